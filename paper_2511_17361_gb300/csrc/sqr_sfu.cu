// sqr_sfu.cu -- sq_measure_sfu: the measured throughput of the special-function
// unit (the MUFU instructions ex2.approx, lg2.approx, rcp.approx), the unit that
// bounds the renderer's pair kernels (9 MUFU per pair in the forward, 13 in the
// backward).  A diagnostic with no counterpart in the paper: the roofline the
// benchmark reports divides by this measured rate rather than by a nominal
// count per clock.
//
// Every thread runs NCH independent chains x <- mufu(x) (a sign or an FP32 add
// per step keeps x in a bounded range), so the unit, not the chains' latency,
// sets the rate.  The results feed a comparison against a value no
// chain reaches, so the compiler keeps the work; nothing is written in practice.
#include "sqr_render.cuh"

namespace sqr {

namespace {

constexpr int NCH = 8;
constexpr int SFU_THREADS = 256;

__device__ float g_sfu_sink;

template <int OP>
__global__ void __launch_bounds__(SFU_THREADS) k_sfu(int iters) {
    float x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = 0.25f + 0.001f * (float)((threadIdx.x + 37 * c) & 255);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            if (OP == 0) x[c] = ex2(-x[c]);        // x in (0, 1]: 2^-x in [1/2, 1)
            if (OP == 1) x[c] = lg2(x[c] + 2.f);   // x + 2 in [2, 4): log2 in [1, 2)
            if (OP == 2) x[c] = rcp(x[c] + 1.f);   // x + 1 in [1, 2]: 1/(x+1) in [1/2, 1]
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    if (s == -1.f) g_sfu_sink = s;  // never true: every chain stays positive
}

}  // namespace

}  // namespace sqr

extern "C" sq_status_t sq_measure_sfu(int op, double* ops_per_s, void* stream) {
    using namespace sqr;
    if (!ops_per_s || op < 0 || op > 2) {
        set_last_error("sq_measure_sfu: op must be 0 (ex2), 1 (lg2) or 2 (rcp) and ops_per_s non-NULL");
        return SQ_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const void* fn = op == 0 ? (const void*)k_sfu<0> : op == 1 ? (const void*)k_sfu<1> : (const void*)k_sfu<2>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SFU_THREADS, 0);
    if (e != cudaSuccess) return cuda_status(e, "sq_measure_sfu occupancy");
    const int blocks = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    const int iters = 4096;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_status(e, "sq_measure_sfu event");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_status(e, "sq_measure_sfu event");
    }
    void* args[] = {(void*)&iters};
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up; the fastest counts
        cudaEventRecord(e0, st);
        e = cudaLaunchKernel(fn, dim3(blocks), dim3(SFU_THREADS), args, 0, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e, "sq_measure_sfu");
    *ops_per_s = (double)blocks * SFU_THREADS * (double)iters * NCH / (best * 1e-3);
    return SQ_OK;
}
