// sqr_common.cuh -- device building blocks shared by the sm_103a kernels of the
// superquadric renderer: grid constants, the FP32 sample/voxel rule, packed
// per-primitive records, hardware exp2/log2, warp helpers and error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sqr.h"

namespace sqr {

constexpr int WARP = 32;
constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;

// ---------------------------------------------------------------- host errors
void set_last_error(const char* fmt, ...);
sq_status_t cuda_status(cudaError_t e, const char* where);
#define SQ_CHECK_LAUNCH(where)                                 \
    do {                                                       \
        cudaError_t _e = cudaGetLastError();                   \
        if (_e != cudaSuccess) return cuda_status(_e, where);  \
    } while (0)

// Optional per-kernel timing (sq_profile_enable): events on the launching stream
// around every launch of the library.
void prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);

// A <<<...>>> launch of kernel `name`, timed when profiling is on, then checked.
#define SQ_LAUNCH(name, st, ...)       \
    do {                               \
        ::sqr::prof_begin(name, st);   \
        __VA_ARGS__;                   \
        ::sqr::prof_end(st);           \
        SQ_CHECK_LAUNCH(name);         \
    } while (0)

// ---------------------------------------------------------------- bounds checks
// Debug build (-DSQR_CHECK, libsqr_check.so): SQ_BOUND(cond, site) records the first
// failing check of the translation unit in a device word and returns false, and the
// caller skips the access it guards.  No trap, no assert: the kernel goes on, and the
// host reads and clears the words with sq_check_query.  In the normal build it is
// `true` and compiles away.  Sites: 1 a voxel list (V_f, V_n) outside V_sq, 2 a
// listed id that is not a primitive, 3 a saved-state page outside the buffer.
#ifdef SQR_CHECK
static __device__ unsigned int g_check_site;
__device__ __forceinline__ bool check_ok(bool c, unsigned site) {
    if (!c) atomicCAS(&g_check_site, 0u, site);
    return c;
}
static inline unsigned check_take() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_site, sizeof v) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_check_site, &z, sizeof z);
    return v;
}
#define SQ_BOUND(cond, site) ::sqr::check_ok((cond), (site))
#else
#define SQ_BOUND(cond, site) true
#endif

// ---------------------------------------------------------------- grid
struct GridC {
    int n[3];
    float lo[3];
    float inv_vs[3];  // 1.0f / vs (IEEE division on the host)
    float vs[3];
    float nf[3];      // n as float (exact, n < 2^24 per axis)
};

GridC make_grid(const sq_grid_t* g);

// Sample x = o + t d in FP32 (multiply, then add; no contraction) and its voxel
// id, -1 when any axis falls outside [0, n).
__device__ __forceinline__ int sample_voxel(const GridC& g, const float o[3], const float d[3], float t, float x[3],
                                            int idx[3]) {
    bool inside = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        x[i] = __fadd_rn(o[i], __fmul_rn(t, d[i]));
        float u = __fmul_rn(__fsub_rn(x[i], g.lo[i]), g.inv_vs[i]);
        bool in = (u >= 0.0f) && (u < g.nf[i]);
        inside = inside && in;
        idx[i] = in ? (int)floorf(u) : 0;
    }
    return inside ? (idx[0] * g.n[1] + idx[1]) * g.n[2] + idx[2] : -1;
}

__device__ __forceinline__ int sample_voxel(const GridC& g, const float o[3], const float d[3], float t, float x[3]) {
    int idx[3];
    return sample_voxel(g, o, d, t, x, idx);
}

// Pinhole ray through the centre of pixel (u, v): FP32, correctly rounded
// operations in a fixed order (no FMA contraction), so that the sample voxels
// are reproducible on any IEEE machine.
__device__ __forceinline__ void pixel_ray(const float* __restrict__ K, const float* __restrict__ c2w, int u, int v,
                                          float o[3], float d[3]) {
    float a = __fsub_rn(__fadd_rn(__int2float_rn(u), 0.5f), K[2]);
    float dx = __fdiv_rn(a, K[0]);
    float b = __fsub_rn(__fadd_rn(__int2float_rn(v), 0.5f), K[3]);
    float dy = __fdiv_rn(b, K[1]);
    float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), 1.0f);
    float nrm = __fsqrt_rn(n2);
    float cx = __fdiv_rn(dx, nrm), cy = __fdiv_rn(dy, nrm), cz = __fdiv_rn(1.0f, nrm);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float di = __fadd_rn(__fmul_rn(c2w[4 * i + 0], cx), __fmul_rn(c2w[4 * i + 1], cy));
        d[i] = __fadd_rn(di, __fmul_rn(c2w[4 * i + 2], cz));
        o[i] = c2w[4 * i + 3];
    }
}

// ---------------------------------------------------------------- MUFU
// Hardware base-2 exponential / logarithm (SFU).  ex2(-inf) = 0, lg2(0) = -inf.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------- packed primitive
// Forward record, 4 x float4 = 64 B per primitive:
//   r0 = (m.x, m.y, m.z, sigma)
//   r1 = (M0.x, M0.y, M0.z, ea)   M_j = (column j of R) / s_j, so that the scaled
//   r2 = (M1.x, M1.y, M1.z, eb)   canonical coordinate is u_j = M_j . (x - m)
//   r3 = (M2.x, M2.y, M2.z, ec)   ea = 2/eps2, eb = eps2/eps1, ec = 2/eps1
// Backward extras, 3 x float4 = 48 B per primitive:
//   a0 = (qn.w, qn.x, qn.y, qn.z)   normalised quaternion
//   a1 = (1/|q|, 1/s.x, 1/s.y, 1/s.z)
//   a2 = (eps1, eps2, 1/eps1, 1/eps2)
constexpr int REC4 = 4;
constexpr int AUX4 = 3;

struct Prim {
    float m[3];
    float sigma;
    float M[3][3];
    float ea, eb, ec;
};

__device__ __forceinline__ Prim load_prim(const float4* __restrict__ rec, int k) {
    const float4* r = rec + (size_t)k * REC4;
    float4 r0 = __ldg(r + 0), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
    Prim p;
    p.m[0] = r0.x; p.m[1] = r0.y; p.m[2] = r0.z; p.sigma = r0.w;
    p.M[0][0] = r1.x; p.M[0][1] = r1.y; p.M[0][2] = r1.z; p.ea = r1.w;
    p.M[1][0] = r2.x; p.M[1][1] = r2.y; p.M[1][2] = r2.z; p.eb = r2.w;
    p.M[2][0] = r3.x; p.M[2][1] = r3.y; p.M[2][2] = r3.z; p.ec = r3.w;
    return p;
}

// Occupancy (Eq. 1-2) of primitive p at point x: exp(-f(x_S)) evaluated with
// the SFU: a^e = 2^(e log2 a).  Zero bases give -inf logs and 0 powers; far
// points give f = inf and p = 0, never NaN.
__device__ __forceinline__ float occupancy(const Prim& p, const float x[3]) {
    float d0 = x[0] - p.m[0], d1 = x[1] - p.m[1], d2 = x[2] - p.m[2];
    float u0 = fmaf(p.M[0][0], d0, fmaf(p.M[0][1], d1, p.M[0][2] * d2));
    float u1 = fmaf(p.M[1][0], d0, fmaf(p.M[1][1], d1, p.M[1][2] * d2));
    float u2 = fmaf(p.M[2][0], d0, fmaf(p.M[2][1], d1, p.M[2][2] * d2));
    float pa = ex2(p.ea * lg2(fabsf(u0)));
    float pb = ex2(p.ea * lg2(fabsf(u1)));
    float pc = ex2(p.ec * lg2(fabsf(u2)));
    float PA = ex2(p.eb * lg2(pa + pb));
    return ex2(-(PA + pc) * LOG2E);
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Inclusive product scan across the warp.
__device__ __forceinline__ float warp_incl_prod(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v *= y;
    }
    return v;
}

__device__ __forceinline__ void red_add(float* addr, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(v) : "memory");
}

// Packs S into the forward and backward records (host launcher in sqr_render.cu).
sq_status_t launch_pack(const sq_prims_t* prims, float4* rec, float4* aux, float* logits_pad, int cp,
                        cudaStream_t st);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
inline int cpad(int c) { return (c + 3) / 4 * 4; }

// Host-side argument checks shared by the entry points.
sq_status_t check_prims(const sq_prims_t* p);
sq_status_t check_grid(const sq_grid_t* g);
sq_status_t check_index(const sq_index_t* idx, const sq_grid_t* g, int n);
sq_status_t check_rays(const sq_rays_t* r);

}  // namespace sqr
