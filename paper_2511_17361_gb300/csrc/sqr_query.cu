// sqr_query.cu -- voxelisation of Supp. A.4 through the same index: at every
// voxel centre p, density = sum_{k in Q(v)} p_o(p, S_k) sigma_k and the semantic
// sum s = sum p_o c_k; label = argmax_c s (lowest index on ties) when density >= tau,
// otherwise "free" (= C).
//
// One thread per voxel (voxel ids are z-fastest, so a warp covers neighbouring
// voxels with near-identical lists and the primitive gathers hit L1).  The
// per-voxel semantic row is staged in shared memory so that the [nvox, C] output
// is written with coalesced stores.
#include "sqr_common.cuh"

namespace sqr {

namespace {

constexpr int Q_THREADS = 128;

struct QueryArgs {
    const float4* rec;
    const float* lpad;
    const int* v_n;
    const int* v_f;
    const int* v_sq;
    const int* status;
    GridC g;
    long long nvox;
    int C;
    float tau;
    float* density;
    float* sem;
    unsigned char* label;
};

template <int CP>
__global__ void __launch_bounds__(Q_THREADS) k_query(QueryArgs a) {
    __shared__ float rows[Q_THREADS * (CP + 1)];
    if (*a.status != SQ_OK) return;
    const float4* lp4 = reinterpret_cast<const float4*>(a.lpad);
    const int ny = a.g.n[1], nz = a.g.n[2];
    for (long long base = (long long)blockIdx.x * Q_THREADS; base < a.nvox; base += (long long)gridDim.x * Q_THREADS) {
        const long long v = base + threadIdx.x;
        float acc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = 0.f;
        if (v < a.nvox) {
            const int iz = (int)(v % nz);
            const int iy = (int)((v / nz) % ny);
            const int ix = (int)(v / ((long long)ny * nz));
            const int id[3] = {ix, iy, iz};
            float x[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                x[i] = __fadd_rn(a.g.lo[i], __fmul_rn(__fadd_rn(__int2float_rn(id[i]), 0.5f), a.g.vs[i]));
            const int n = __ldg(a.v_n + v), f = __ldg(a.v_f + v);
            float dens = 0.f;
            for (int e = 0; e < n; ++e) {
                const int k = __ldg(a.v_sq + f + e);
                Prim p = load_prim(a.rec, k);
                const float po = occupancy(p, x);
                dens = fmaf(po, p.sigma, dens);
                const float4* cr = lp4 + (size_t)k * (CP / 4);
#pragma unroll
                for (int q = 0; q < CP / 4; ++q) {
                    float4 cv = __ldg(cr + q);
                    acc[4 * q + 0] = fmaf(po, cv.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(po, cv.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(po, cv.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(po, cv.w, acc[4 * q + 3]);
                }
            }
            a.density[v] = dens;
            if (a.label) {
                int best = 0;
                float bv = acc[0];
#pragma unroll
                for (int c = 1; c < CP; ++c)
                    if (c < a.C && acc[c] > bv) {
                        bv = acc[c];
                        best = c;
                    }
                a.label[v] = (unsigned char)(dens >= a.tau ? best : a.C);
            }
        }
#pragma unroll
        for (int c = 0; c < CP; ++c) rows[threadIdx.x * (CP + 1) + c] = acc[c];
        __syncthreads();
        const long long nrow = (a.nvox - base) < Q_THREADS ? (a.nvox - base) : Q_THREADS;
        const long long total = nrow * a.C;
        float* out = a.sem + base * a.C;
        for (long long e = threadIdx.x; e < total; e += Q_THREADS) {
            const int row = (int)(e / a.C), c = (int)(e - (long long)row * a.C);
            out[e] = rows[row * (CP + 1) + c];
        }
        __syncthreads();
    }
}

}  // namespace

size_t render_workspace_size(const sq_prims_t* p);

template <int CP>
static sq_status_t launch_query_cp(const QueryArgs& a, cudaStream_t st) {
    long long want = (a.nvox + Q_THREADS - 1) / Q_THREADS;
    int blocks = (int)(want < 152LL * 64 ? want : 152LL * 64);
    if (blocks < 1) blocks = 1;
    SQ_LAUNCH("k_query", st, k_query<CP><<<blocks, Q_THREADS, 0, st>>>(a));
    return SQ_OK;
}

sq_status_t query_grid_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid, float tau,
                            float* density, float* sem, unsigned char* label, void* ws, size_t ws_bytes,
                            cudaStream_t st) {
    size_t need = render_workspace_size(prims);
    if (ws == nullptr || ws_bytes < need) {
        set_last_error("sq_query_grid: workspace of %zu bytes given, %zu needed", ws_bytes, need);
        return SQ_ERR_INVALID_ARG;
    }
    const int cp = cpad(prims->n_classes);
    // packed records at the start of the workspace, padded logits after them
    char* base = (char*)ws;
    float4* rec = (float4*)base;
    float* lpad = (float*)(base + align_up((size_t)prims->n * REC4 * sizeof(float4), 256));
    sq_status_t s = launch_pack(prims, rec, nullptr, lpad, cp, st);
    if (s != SQ_OK) return s;
    QueryArgs a;
    a.rec = rec;
    a.lpad = lpad;
    a.v_n = idx->v_n;
    a.v_f = idx->v_f;
    a.v_sq = idx->v_sq;
    a.status = idx->status;
    a.g = make_grid(grid);
    a.nvox = (long long)grid->nx * grid->ny * grid->nz;
    a.C = prims->n_classes;
    a.tau = tau;
    a.density = density;
    a.sem = sem;
    a.label = label;
    switch (cp) {
        case 4: return launch_query_cp<4>(a, st);
        case 8: return launch_query_cp<8>(a, st);
        case 12: return launch_query_cp<12>(a, st);
        case 16: return launch_query_cp<16>(a, st);
        case 20: return launch_query_cp<20>(a, st);
        case 24: return launch_query_cp<24>(a, st);
        case 28: return launch_query_cp<28>(a, st);
        case 32: return launch_query_cp<32>(a, st);
        default: return SQ_ERR_INVALID_ARG;
    }
}

}  // namespace sqr
