// sqr_api.cu -- the extern "C" entry points declared in include/sqr.h: host-side
// argument validation, workspace sizing, status strings, and the training-loss
// kernel (Supp. A.5, Eq. 8) used to drive the backward pass.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "sqr_common.cuh"
#include "sqr_render.cuh"

namespace sqr {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

sq_status_t cuda_status(cudaError_t e, const char* where) {
    set_last_error("%s: %s", where, cudaGetErrorString(e));
    return SQ_ERR_CUDA;
}

GridC make_grid(const sq_grid_t* g) {
    GridC c;
    c.n[0] = g->nx; c.n[1] = g->ny; c.n[2] = g->nz;
    for (int i = 0; i < 3; ++i) {
        c.lo[i] = g->lo[i];
        c.vs[i] = g->vs[i];
        c.inv_vs[i] = 1.0f / g->vs[i];
        c.nf[i] = (float)c.n[i];
    }
    return c;
}

sq_status_t check_prims(const sq_prims_t* p) {
    if (!p) { set_last_error("prims is NULL"); return SQ_ERR_INVALID_ARG; }
    if (p->n < 0) { set_last_error("prims.n = %d < 0", p->n); return SQ_ERR_INVALID_ARG; }
    if (p->n_classes < 1 || p->n_classes > SQ_MAX_CLASSES) {
        set_last_error("prims.n_classes = %d outside [1, %d]", p->n_classes, SQ_MAX_CLASSES);
        return SQ_ERR_INVALID_ARG;
    }
    if (p->n > 0 && (!p->means || !p->quats || !p->scales || !p->eps || !p->opacity || !p->logits)) {
        set_last_error("a primitive parameter pointer is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    if (p->sem_mode != SQ_SEM_RAW && p->sem_mode != SQ_SEM_SOFTMAX) {
        set_last_error("prims.sem_mode = %d unknown", p->sem_mode);
        return SQ_ERR_INVALID_ARG;
    }
    return SQ_OK;
}

sq_status_t check_grid(const sq_grid_t* g) {
    if (!g) { set_last_error("grid is NULL"); return SQ_ERR_INVALID_ARG; }
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nx > (1 << 24) || g->ny > (1 << 24) || g->nz > (1 << 24)) {
        set_last_error("grid dims (%d, %d, %d) invalid", g->nx, g->ny, g->nz);
        return SQ_ERR_INVALID_ARG;
    }
    long long nvox = (long long)g->nx * g->ny * g->nz;
    long long ndiff = (long long)(g->nx + 1) * (g->ny + 1) * (g->nz + 1);
    if (nvox >= 2147483647LL || ndiff >= 2147483647LL) {
        set_last_error("grid has %lld voxels, at most 2^31 - 1 supported", nvox);
        return SQ_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3; ++i) {
        if (!(g->vs[i] > 0.f) || !isfinite(g->vs[i]) || !isfinite(g->lo[i])) {
            set_last_error("grid lo/vs invalid on axis %d", i);
            return SQ_ERR_INVALID_ARG;
        }
    }
    return SQ_OK;
}

sq_status_t check_index(const sq_index_t* idx, const sq_grid_t* g, int n) {
    (void)g;
    if (!idx) { set_last_error("index is NULL"); return SQ_ERR_INVALID_ARG; }
    if (!idx->v_n || !idx->v_f || !idx->status || !idx->p_total || (n > 0 && !idx->ranges)) {
        set_last_error("an index buffer pointer is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    if (idx->capacity < 0) { set_last_error("index capacity < 0"); return SQ_ERR_INVALID_ARG; }
    if (idx->capacity > 0 && !idx->v_sq) { set_last_error("index v_sq is NULL"); return SQ_ERR_INVALID_ARG; }
    return SQ_OK;
}

sq_status_t check_rays(const sq_rays_t* r) {
    if (!r) { set_last_error("rays is NULL"); return SQ_ERR_INVALID_ARG; }
    if (r->n_cam < 0 || r->H < 0 || r->W < 0) {
        set_last_error("rays dims (%d, %d, %d) invalid", r->n_cam, r->H, r->W);
        return SQ_ERR_INVALID_ARG;
    }
    if (r->L < 1 || r->L > SQ_MAX_SAMPLES) {
        set_last_error("rays.L = %d outside [1, %d]", r->L, SQ_MAX_SAMPLES);
        return SQ_ERR_INVALID_ARG;
    }
    if ((long long)r->n_cam * r->H * r->W > 0 && (!r->K || !r->cam2world || !r->t)) {
        set_last_error("a camera pointer is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    if (!(r->kappa >= 0.f && r->kappa < 1.f) || !(r->alpha_max > 0.f) || !isfinite(r->alpha_max)) {
        set_last_error("kappa must be in [0, 1) and alpha_max > 0");
        return SQ_ERR_INVALID_ARG;
    }
    return SQ_OK;
}

size_t index_workspace_size(const sq_grid_t* g);
size_t render_workspace_size(const sq_prims_t* p);
size_t query_workspace_size(const sq_prims_t* p, const sq_grid_t* g);
size_t render_bwd_workspace_size(const sq_prims_t* p, const sq_rays_t* r);
sq_status_t build_index_impl(const sq_prims_t*, const sq_grid_t*, const sq_index_opts_t*, sq_index_t*, void*, size_t,
                             cudaStream_t);
sq_status_t render_fwd_impl(const sq_prims_t*, const sq_index_t*, const sq_grid_t*, const sq_rays_t*, float*, float*,
                            float*, void*, size_t, void*, size_t, cudaStream_t);
sq_status_t render_bwd_impl(const sq_prims_t*, const sq_index_t*, const sq_grid_t*, const sq_rays_t*, const void*,
                            size_t, const float*, const float*, float*, float*, float*, float*, float*, float*, void*,
                            size_t, cudaStream_t);
size_t saved_size(const sq_rays_t* r, int n_classes);
size_t saved_size_pages(const sq_rays_t* r, int n_classes, long long pages);
sq_status_t query_grid_bwd_impl(const sq_prims_t*, const sq_index_t*, const sq_grid_t*, const float*, const float*,
                                float*, float*, float*, float*, float*, float*, void*, size_t, cudaStream_t);
sq_status_t query_grid_impl(const sq_prims_t*, const sq_index_t*, const sq_grid_t*, float, float*, float*,
                            unsigned char*, void*, size_t, cudaStream_t);
sq_status_t count_pairs_impl(const sq_index_t*, const sq_grid_t*, const sq_rays_t*, long long*, cudaStream_t);
size_t batched_workspace_size(const sq_scene_t* scenes, int n);
sq_status_t batched_api_impl(int op, const sq_scene_t* sc, int n, const sq_tuning_t* tuning, void* ws, size_t ws_bytes,
                             cudaStream_t st);
sq_status_t autotune_impl(const sq_scene_t* sc, int n, void* ws, size_t ws_bytes, cudaStream_t st, sq_tuning_t* best,
                          float* fwd_ms, float* bwd_ms, int reps);

// Host checks of every scene of a batch.
static sq_status_t check_scenes(const sq_scene_t* sc, int n) {
    if (!sc || n < 1 || n > SQ_MAX_BATCH) {
        set_last_error("scenes: %d scenes, 1..%d supported", n, SQ_MAX_BATCH);
        return SQ_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        sq_status_t s;
        if ((s = check_prims(&sc[i].prims)) != SQ_OK) return s;
        if ((s = check_grid(&sc[i].grid)) != SQ_OK) return s;
        if ((s = check_index(&sc[i].index, &sc[i].grid, sc[i].prims.n)) != SQ_OK) return s;
        if ((s = check_rays(&sc[i].rays)) != SQ_OK) return s;
    }
    return SQ_OK;
}

// ------------------------------------------------------------------ loss
namespace {
constexpr int LOSS_THREADS = 256;

constexpr int LOSS_WARPS = LOSS_THREADS / 32;

// The n = rows * C floats of `rows` consecutive rows of a row-major [*, C] array
// (C <= 32) to and from a warp's shared-memory block of 32 rows of stride sp, with
// coalesced global accesses: lane l takes flat indices i = l + 32 k, row i / C,
// column i % C, stepped as a mixed-radix sum (no division in the loop).
__device__ __forceinline__ void rows_in(float* buf, const float* __restrict__ src, int n, int C, int sp, int lane) {
    int row = lane / C, col = lane % C;
    const int drow = 32 / C, dcol = 32 % C;
    for (int i = lane; i < n; i += 32) {
        buf[row * sp + col] = __ldg(src + i);
        row += drow;
        col += dcol;
        if (col >= C) {
            col -= C;
            ++row;
        }
    }
}

__device__ __forceinline__ void rows_out(float* __restrict__ dst, const float* buf, int n, int C, int sp, int lane) {
    int row = lane / C, col = lane % C;
    const int drow = 32 / C, dcol = 32 % C;
    for (int i = lane; i < n; i += 32) {
        dst[i] = buf[row * sp + col];
        row += drow;
        col += dcol;
        if (col >= C) {
            col -= C;
            ++row;
        }
    }
}

// A warp takes 32 consecutive rays at a time: their semantic rows are read into
// shared memory with coalesced loads (rows_in), each lane computes its ray's
// softmax cross-entropy and gradient row there (row stride C | 1 words, so the
// lanes' rows fall in distinct banks), and the gradient rows leave with coalesced
// stores (rows_out).  Per class one expf, as the gradient reuses the softmax numerators.  A
// label outside [0, C) makes that ray's loss NaN and adds no one-hot term.
__global__ void __launch_bounds__(LOSS_THREADS) k_loss(const float* __restrict__ depth, const float* __restrict__ sem,
                                                       const float* __restrict__ td, const int* __restrict__ lab,
                                                       long long R, int C, float ws, float wd, float* __restrict__ loss,
                                                       float* __restrict__ gd, float* __restrict__ gs) {
    extern __shared__ float lrows[];  // [LOSS_WARPS][32][C | 1]
    __shared__ float red[LOSS_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int sp = C | 1;
    float* buf = lrows + (size_t)wid * 32 * sp;
    float part = 0.f;
    const long long nchunk = (R + 31) / 32;
    for (long long ch = (long long)blockIdx.x * LOSS_WARPS + wid; ch < nchunk; ch += (long long)gridDim.x * LOSS_WARPS) {
        const long long r0 = ch * 32;
        const int n = (int)min(32LL, R - r0) * C;
        rows_in(buf, sem + r0 * C, n, C, sp, lane);
        __syncwarp();
        const long long r = r0 + lane;
        if (r < R) {
            float* sr = buf + lane * sp;
            float mx = sr[0];
            for (int c = 1; c < C; ++c) mx = fmaxf(mx, sr[c]);
            const int y = lab[r];
            const bool yok = y >= 0 && y < C;
            const float sy = yok ? sr[y] : __int_as_float(0x7fc00000);
            float z = 0.f;
            for (int c = 0; c < C; ++c) {
                const float e = expf(sr[c] - mx);
                sr[c] = e;
                z += e;
            }
            const float ce = mx + logf(z) - sy;
            const float iz = 1.f / z;
            for (int c = 0; c < C; ++c) sr[c] = ws * (sr[c] * iz - (c == y ? 1.f : 0.f));
            const float diff = depth[r] - td[r];
            gd[r] = wd * 2.f * diff;
            part += ws * ce + wd * diff * diff;
        }
        __syncwarp();
        rows_out(gs + r0 * C, buf, n, C, sp, lane);
        __syncwarp();
    }
    part = warp_sum(part);
    if (lane == 0) red[wid] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < LOSS_WARPS ? red[threadIdx.x] : 0.f;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(loss, v);
    }
}
// Voxel losses: counts of occupied / labelled voxels (first kernel), then the
// losses and gradients normalised by them (second kernel).
__global__ void __launch_bounds__(LOSS_THREADS) k_vloss_count(const int* __restrict__ lab, long long V, int C,
                                                              int* __restrict__ counts) {
    int no = 0, nl = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const int y = lab[v];
        no += (y >= 0 && y < C) ? 1 : 0;
        nl += (y >= 0 && y <= C) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        no += __shfl_xor_sync(0xffffffffu, no, o);
        nl += __shfl_xor_sync(0xffffffffu, nl, o);
    }
    if ((threadIdx.x & 31) == 0 && (no || nl)) {
        atomicAdd(counts, no);
        atomicAdd(counts + 1, nl);
    }
}

// Rows of 32 voxels at a time through shared memory, as k_loss does.
__global__ void __launch_bounds__(LOSS_THREADS) k_vloss(const float* __restrict__ dens, const float* __restrict__ sem,
                                                        const int* __restrict__ lab, long long V, int C, float ls,
                                                        float lo, const int* __restrict__ counts,
                                                        float* __restrict__ loss, float* __restrict__ gd,
                                                        float* __restrict__ gs) {
    extern __shared__ float lrows[];  // [LOSS_WARPS][32][C | 1]
    __shared__ float red[2][LOSS_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int sp = C | 1;
    float* buf = lrows + (size_t)wid * 32 * sp;
    const int no = counts[0], nl = counts[1];
    const float ws = no > 0 ? ls / (float)no : 0.f, wo = nl > 0 ? lo / (float)nl : 0.f;
    float pce = 0.f, pbce = 0.f;
    const long long nchunk = (V + 31) / 32;
    for (long long ch = (long long)blockIdx.x * LOSS_WARPS + wid; ch < nchunk; ch += (long long)gridDim.x * LOSS_WARPS) {
        const long long v0 = ch * 32;
        const int n = (int)min(32LL, V - v0) * C;
        rows_in(buf, sem + v0 * C, n, C, sp, lane);
        __syncwarp();
        const long long v = v0 + lane;
        if (v < V) {
            const int y = lab[v];
            float* sr = buf + lane * sp;
            if (y >= 0 && y < C) {  // cross-entropy of the class probabilities
                float mx = sr[0];
                for (int c = 1; c < C; ++c) mx = fmaxf(mx, sr[c]);
                const float sy = sr[y];
                float z = 0.f;
                for (int c = 0; c < C; ++c) {
                    const float e = expf(sr[c] - mx);
                    sr[c] = e;
                    z += e;
                }
                pce += mx + logf(z) - sy;
                const float iz = 1.f / z;
                for (int c = 0; c < C; ++c) sr[c] = ws * (sr[c] * iz - (c == y ? 1.f : 0.f));
            } else {
                for (int c = 0; c < C; ++c) sr[c] = 0.f;
            }
            const float d = fmaxf(dens[v], 0.f);
            float gdv = 0.f;
            if (y == C) {  // free: -log(1 - p) = d
                pbce += d;
                gdv = dens[v] > 0.f ? wo : 0.f;
            } else if (y >= 0 && y < C) {  // occupied: -log p
                const float dc = fmaxf(d, 1e-6f);
                pbce += -logf(-expm1f(-dc));
                gdv = d > 1e-6f ? -wo / expm1f(dc) : 0.f;
            }
            gd[v] = gdv;
        }
        __syncwarp();
        rows_out(gs + v0 * C, buf, n, C, sp, lane);
        __syncwarp();
    }
    pce = warp_sum(pce);
    pbce = warp_sum(pbce);
    if (lane == 0) {
        red[0][wid] = pce;
        red[1][wid] = pbce;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float a = threadIdx.x < LOSS_WARPS ? red[0][threadIdx.x] : 0.f;
        float b = threadIdx.x < LOSS_WARPS ? red[1][threadIdx.x] : 0.f;
        a = warp_sum(a) * ws;
        b = warp_sum(b) * wo;
        if (threadIdx.x == 0) {
            atomicAdd(loss, a + b);
            atomicAdd(loss + 1, a);
            atomicAdd(loss + 2, b);
        }
    }
}
}  // namespace

}  // namespace sqr

using namespace sqr;

#ifdef SQR_CHECK
namespace sqr {
unsigned check_take_fwd();
unsigned check_take_bwd();
unsigned check_take_query();
}  // namespace sqr
#endif

extern "C" {

const char* sq_status_string(sq_status_t s) {
    switch (s) {
        case SQ_OK: return "SQ_OK";
        case SQ_ERR_INVALID_ARG: return "SQ_ERR_INVALID_ARG: invalid argument";
        case SQ_ERR_CAPACITY: return "SQ_ERR_CAPACITY: index entries exceed the v_sq capacity";
        case SQ_ERR_CUDA: return "SQ_ERR_CUDA: CUDA error";
        case SQ_ERR_TIMEOUT: return "SQ_ERR_TIMEOUT: bounded device wait expired";
        case SQ_ERR_NUMERIC: return "SQ_ERR_NUMERIC: a superquadric parameter outside its domain";
    }
    return "unknown status";
}

const char* sq_last_error(void) { return g_last_error; }

size_t sq_workspace_size(int op, const sq_prims_t* prims, const sq_grid_t* grid, const sq_rays_t* rays) {
    switch (op) {
        case SQ_OP_INDEX:
            if (check_grid(grid) != SQ_OK) return 0;
            return index_workspace_size(grid);
        case SQ_OP_FWD:
            if (check_prims(prims) != SQ_OK) return 0;
            return render_workspace_size(prims);
        case SQ_OP_QUERY:
            if (check_prims(prims) != SQ_OK || check_grid(grid) != SQ_OK) return 0;
            return query_workspace_size(prims, grid);
        case SQ_OP_BWD:
            if (check_prims(prims) != SQ_OK || check_rays(rays) != SQ_OK) return 0;
            return render_bwd_workspace_size(prims, rays);
    }
    set_last_error("sq_workspace_size: unknown op %d", op);
    return 0;
}

sq_status_t sq_build_index(const sq_prims_t* prims, const sq_grid_t* grid, const sq_index_opts_t* opts,
                           sq_index_t* index, void* ws, size_t ws_bytes, void* stream) {
    sq_status_t s;
    if ((s = check_prims(prims)) != SQ_OK) return s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, prims->n)) != SQ_OK) return s;
    if (!opts) { set_last_error("opts is NULL"); return SQ_ERR_INVALID_ARG; }
    if (opts->mode == SQ_INDEX_OBB || opts->mode == SQ_INDEX_OBB_OPACITY) {
        if (!(opts->tau_cut > 0.f && opts->tau_cut < 1.f)) {
            set_last_error("tau_cut = %g outside (0, 1)", (double)opts->tau_cut);
            return SQ_ERR_INVALID_ARG;
        }
    } else if (opts->mode == SQ_INDEX_CUBE) {
        if (opts->nv < 0 || opts->nv > (1 << 20)) { set_last_error("nv = %d invalid", opts->nv); return SQ_ERR_INVALID_ARG; }
    } else {
        set_last_error("index mode %d unknown", opts->mode);
        return SQ_ERR_INVALID_ARG;
    }
    return build_index_impl(prims, grid, opts, index, ws, ws_bytes, (cudaStream_t)stream);
}

size_t sq_saved_size(const sq_rays_t* rays, int n_classes) {
    if (check_rays(rays) != SQ_OK) return 0;
    if (n_classes < 1 || n_classes > SQ_MAX_CLASSES) {
        set_last_error("n_classes = %d outside 1..%d", n_classes, SQ_MAX_CLASSES);
        return 0;
    }
    return saved_size(rays, n_classes);
}

size_t sq_saved_size_pages(const sq_rays_t* rays, int n_classes, long long pages) {
    if (check_rays(rays) != SQ_OK) return 0;
    if (n_classes < 1 || n_classes > SQ_MAX_CLASSES || pages < 1) {
        set_last_error("n_classes = %d outside 1..%d or pages = %lld < 1", n_classes, SQ_MAX_CLASSES, pages);
        return 0;
    }
    return saved_size_pages(rays, n_classes, pages);
}

sq_status_t sq_render_fwd(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                          const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* saved,
                          size_t saved_bytes, void* ws, size_t ws_bytes, void* stream) {
    sq_status_t s;
    if ((s = check_prims(prims)) != SQ_OK) return s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, prims->n)) != SQ_OK) return s;
    if ((s = check_rays(rays)) != SQ_OK) return s;
    if ((long long)rays->n_cam * rays->H * rays->W > 0 && (!depth || !sem)) {
        set_last_error("sq_render_fwd: depth/sem output is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    return render_fwd_impl(prims, index, grid, rays, depth, sem, t_final, saved, saved_bytes, ws, ws_bytes,
                           (cudaStream_t)stream);
}

sq_status_t sq_render_bwd(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                          const sq_rays_t* rays, const void* saved, size_t saved_bytes, const float* grad_depth,
                          const float* grad_sem, float* g_means,
                          float* g_quats, float* g_scales, float* g_eps, float* g_opacity, float* g_logits, void* ws,
                          size_t ws_bytes, void* stream) {
    sq_status_t s;
    if ((s = check_prims(prims)) != SQ_OK) return s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, prims->n)) != SQ_OK) return s;
    if ((s = check_rays(rays)) != SQ_OK) return s;
    if ((long long)rays->n_cam * rays->H * rays->W > 0 && (!grad_depth || !grad_sem)) {
        set_last_error("sq_render_bwd: grad_depth/grad_sem is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    if (prims->n > 0 && (!g_means || !g_quats || !g_scales || !g_eps || !g_opacity || !g_logits)) {
        set_last_error("sq_render_bwd: a gradient output is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    return render_bwd_impl(prims, index, grid, rays, saved, saved_bytes, grad_depth, grad_sem, g_means, g_quats,
                           g_scales, g_eps, g_opacity, g_logits, ws, ws_bytes, (cudaStream_t)stream);
}

sq_status_t sq_query_grid(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid, float tau,
                          float* density, float* sem, unsigned char* label, void* ws, size_t ws_bytes, void* stream) {
    sq_status_t s;
    if ((s = check_prims(prims)) != SQ_OK) return s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, prims->n)) != SQ_OK) return s;
    if (!density || !sem) { set_last_error("sq_query_grid: output is NULL"); return SQ_ERR_INVALID_ARG; }
    if (label && prims->n_classes > 255) { set_last_error("labels need n_classes <= 255"); return SQ_ERR_INVALID_ARG; }
    return query_grid_impl(prims, index, grid, tau, density, sem, label, ws, ws_bytes, (cudaStream_t)stream);
}

sq_status_t sq_query_grid_bwd(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                              const float* grad_density, const float* grad_sem, float* g_means, float* g_quats,
                              float* g_scales, float* g_eps, float* g_opacity, float* g_logits, void* ws,
                              size_t ws_bytes, void* stream) {
    sq_status_t s;
    if ((s = check_prims(prims)) != SQ_OK) return s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, prims->n)) != SQ_OK) return s;
    if (!grad_density || !grad_sem) {
        set_last_error("sq_query_grid_bwd: a cotangent is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    if (prims->n > 0 && (!g_means || !g_quats || !g_scales || !g_eps || !g_opacity || !g_logits)) {
        set_last_error("sq_query_grid_bwd: a gradient output is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    return query_grid_bwd_impl(prims, index, grid, grad_density, grad_sem, g_means, g_quats, g_scales, g_eps,
                               g_opacity, g_logits, ws, ws_bytes, (cudaStream_t)stream);
}

sq_status_t sq_loss_ce_mse(const float* depth, const float* sem, const float* target_depth, const int* target_label,
                           long long n_rays, int n_classes, float lambda_s, float lambda_d, float* loss,
                           float* grad_depth, float* grad_sem, void* stream) {
    if (n_rays < 0 || n_classes < 1) { set_last_error("sq_loss_ce_mse: bad sizes"); return SQ_ERR_INVALID_ARG; }
    if (!loss || (n_rays > 0 && (!depth || !sem || !target_depth || !target_label || !grad_depth || !grad_sem))) {
        set_last_error("sq_loss_ce_mse: NULL pointer");
        return SQ_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "memset loss");
    if (n_rays == 0) return SQ_OK;
    const float ws = lambda_s / (float)n_rays, wd = lambda_d / (float)n_rays;
    if (n_classes > SQ_MAX_CLASSES) {
        set_last_error("sq_loss_ce_mse: %d classes, at most %d", n_classes, SQ_MAX_CLASSES);
        return SQ_ERR_INVALID_ARG;
    }
    const long long chunks = (n_rays + 31) / 32, want = (chunks + LOSS_WARPS - 1) / LOSS_WARPS;
    const int blocks = (int)(want < (long long)device_sm_count() * 8 ? want : (long long)device_sm_count() * 8);
    const size_t smem = (size_t)LOSS_WARPS * 32 * (n_classes | 1) * sizeof(float);
    SQ_LAUNCH("k_loss", st, k_loss<<<blocks, LOSS_THREADS, smem, st>>>(depth, sem, target_depth, target_label, n_rays,
                                                                      n_classes, ws, wd, loss, grad_depth, grad_sem));
    return SQ_OK;
}

sq_status_t sq_loss_voxel(const float* density, const float* sem, const int* label, long long n_voxels,
                          int n_classes, float lambda_s, float lambda_o, float* loss, int* counts,
                          float* grad_density, float* grad_sem, void* stream) {
    if (n_voxels < 0 || n_classes < 1) { set_last_error("sq_loss_voxel: bad sizes"); return SQ_ERR_INVALID_ARG; }
    if (!loss || !counts || (n_voxels > 0 && (!density || !sem || !label || !grad_density || !grad_sem))) {
        set_last_error("sq_loss_voxel: NULL pointer");
        return SQ_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(loss, 0, 3 * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "memset loss");
    e = cudaMemsetAsync(counts, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e, "memset counts");
    if (n_voxels == 0) return SQ_OK;
    if (n_classes > SQ_MAX_CLASSES) {
        set_last_error("sq_loss_voxel: %d classes, at most %d", n_classes, SQ_MAX_CLASSES);
        return SQ_ERR_INVALID_ARG;
    }
    const long long want = (n_voxels + LOSS_THREADS - 1) / LOSS_THREADS;
    const int blocks = (int)(want < 152LL * 16 ? want : 152LL * 16);
    SQ_LAUNCH("k_vloss_count", st, k_vloss_count<<<blocks, LOSS_THREADS, 0, st>>>(label, n_voxels, n_classes, counts));
    const long long chunks = (n_voxels + 31) / 32, vwant = (chunks + LOSS_WARPS - 1) / LOSS_WARPS;
    const int vblocks = (int)(vwant < (long long)device_sm_count() * 8 ? vwant : (long long)device_sm_count() * 8);
    const size_t smem = (size_t)LOSS_WARPS * 32 * (n_classes | 1) * sizeof(float);
    SQ_LAUNCH("k_vloss", st, k_vloss<<<vblocks, LOSS_THREADS, smem, st>>>(density, sem, label, n_voxels, n_classes,
                                                                        lambda_s, lambda_o, counts, loss,
                                                                        grad_density, grad_sem));
    return SQ_OK;
}

sq_status_t sq_count_pairs(const sq_index_t* index, const sq_grid_t* grid, const sq_rays_t* rays, long long* out,
                           void* stream) {
    sq_status_t s;
    if ((s = check_grid(grid)) != SQ_OK) return s;
    if ((s = check_index(index, grid, 0)) != SQ_OK) return s;
    if ((s = check_rays(rays)) != SQ_OK) return s;
    if (!out) { set_last_error("sq_count_pairs: out is NULL"); return SQ_ERR_INVALID_ARG; }
    return count_pairs_impl(index, grid, rays, out, (cudaStream_t)stream);
}

size_t sq_batched_workspace_size(const sq_scene_t* scenes, int n_scenes) {
    if (check_scenes(scenes, n_scenes) != SQ_OK) return 0;
    return batched_workspace_size(scenes, n_scenes);
}

sq_status_t sq_render_batched(int op, const sq_scene_t* scenes, int n_scenes, const sq_tuning_t* tuning,
                              void* workspace, size_t workspace_bytes, void* stream) {
    sq_status_t s;
    if ((s = check_scenes(scenes, n_scenes)) != SQ_OK) return s;
    if (op != SQ_OP_FWD && op != SQ_OP_BWD) {
        set_last_error("sq_render_batched: op %d is not SQ_OP_FWD or SQ_OP_BWD", op);
        return SQ_ERR_INVALID_ARG;
    }
    return batched_api_impl(op, scenes, n_scenes, tuning, workspace, workspace_bytes, (cudaStream_t)stream);
}

sq_status_t sq_autotune(const sq_scene_t* scenes, int n_scenes, void* workspace, size_t workspace_bytes, void* stream,
                        int reps, sq_tuning_t* best, float* fwd_ms, float* bwd_ms) {
    sq_status_t s;
    if ((s = check_scenes(scenes, n_scenes)) != SQ_OK) return s;
    if (!best) {
        set_last_error("sq_autotune: best is NULL");
        return SQ_ERR_INVALID_ARG;
    }
    return autotune_impl(scenes, n_scenes, workspace, workspace_bytes, (cudaStream_t)stream, best, fwd_ms, bwd_ms,
                         reps);
}

sq_status_t sq_check_query(int* compiled, int* site) {
    if (compiled == nullptr || site == nullptr) {
        sqr::set_last_error("sq_check_query: compiled and site must be non-NULL");
        return SQ_ERR_INVALID_ARG;
    }
#ifdef SQR_CHECK
    unsigned first = 0;
    for (unsigned v : {sqr::check_take_fwd(), sqr::check_take_bwd(), sqr::check_take_query()})
        if (first == 0) first = v;
    *compiled = 1;
    *site = (int)first;
#else
    *compiled = 0;
    *site = 0;
#endif
    return SQ_OK;
}

}  // extern "C"
