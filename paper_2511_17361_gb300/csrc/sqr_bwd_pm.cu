// sqr_bwd_pm.cu -- primitive-major render backward (Sec. 3.3.3, Processes 2-3).
//
// Process 1 (the back-to-front sweep that stores dL/dalpha_j and w_j per sample)
// is shared with the ray-major path.  Here the (sample, superquadric)
// interactions are grouped by primitive, as the paper's Process 2 does, but
// without a sort: the samples whose voxel lies in primitive k's box form, on
// every ray, one interval of consecutive samples (the voxel coordinates of a
// ray's samples are monotone), so the interactions of k are generated directly
// from its box:
//   k_pm_rects  projects the box into every camera: a pixel rectangle that holds
//               every pixel whose ray can meet the box (conservative);
//   k_pm_dirs   the direction and composited sample count of every ray;
//   k_pm_scan   turns the rectangles' pixel counts into tiles (at most PM_MAXT per
//               primitive) and numbers them, with each tile's primitive;
//   k_pm_tiles  (Process 3) persistent blocks (4 per SM) take tiles from a counter:
//               for each candidate pixel a conservative slab test, then the exact
//               sample interval of its ray inside the box (the same FP32
//               sample/voxel rule the forward used: the interval the six plane
//               crossings estimate, accepted when the rule puts its end samples
//               inside the box and their outer neighbours outside, else per-axis
//               searches from the estimates, a binary search as their fallback),
//               then the pass's non-empty runs at their index and its pairs split
//               evenly over the threads, each accumulating the partial derivatives
//               of its pairs; a block reduction writes the tile's sums;
//   k_pm_final  sums each primitive's tiles in tile order into its accumulator.
// Every sum is taken in a fixed order, so the gradients are bitwise reproducible
// (the ray-major path flushes with atomic adds).
#include "sqr_pair.cuh"
#include "sqr_render.cuh"

namespace sqr {

namespace {

constexpr int PM_THREADS = 256;
constexpr int PM_WARPS = PM_THREADS / 32;
constexpr int PM_CPT = PM_CHUNK / PM_THREADS;  // candidates per thread and pass
constexpr int PM_SMCAM = 16;                     // cameras whose rectangles a tile stages in shared memory
constexpr int PM_NS = 2;                         // pairs of one run per walk step (4 and 8 measured slower)
constexpr int PM_CSUB = 4;                       // runs a warp reads gS rows of at once in the class stage
static_assert(PM_CHUNK % PM_THREADS == 0, "whole candidates per thread");
static_assert((PM_CHUNK & (PM_CHUNK - 1)) == 0, "the slot search halves a power of two");

__device__ __forceinline__ int scene_of_prim(const long long* __restrict__ poff, int nsc, int g) {
    int lo = 0, hi = nsc;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(poff + mid) <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int tiles_of(int cnt) {
    constexpr int per = PM_CHUNK * PM_TILE_CHUNKS;
    return cnt <= 0 ? 0 : min(PM_MAXT, (cnt + per - 1) / per);
}

// Pixel rectangle (u0, v0, u1, v1), inclusive, of the pixels whose rays can meet
// the world box [bl, bh] at a sample, for camera (K, c2w) of an H x W image;
// (0, 0, -1, -1) when none can.  Samples lie at t >= t0 along rays through pixel
// centres; in the camera frame (x_cam = R^-1 (x - o)) a sample of pixel (u, v)
// is t (dx, dy, 1) / |(dx, dy, 1)| with dx = (u + 1/2 - cx) / fx, dy likewise,
// so for t0 > 0 its depth is at least zc = t0 / max |(dx, dy, 1)|: the box is
// clipped to the half-space z >= zc / 2 and the vertices of the clipped box
// (corners in front, edge crossings of the plane) are projected.  FP32: its
// rounding is far below the two pixels of margin (the device's FP64 rate made
// this kernel a fifth of a millisecond); degenerate cameras and boxes reaching
// behind a camera whose rays start at t0 <= 0 get the whole image.
__device__ int4 box_rect(const float* __restrict__ K, const float* __restrict__ c2w, int H, int W, const float bl[3],
                         const float bh[3], float t0) {
    const int4 none = make_int4(0, 0, -1, -1), all = make_int4(0, 0, W - 1, H - 1);
    if (W <= 0 || H <= 0) return none;
    const float fx = K[0], fy = K[1], cx = K[2], cy = K[3];
    if (!(fabsf(fx) > 0.f) || !(fabsf(fy) > 0.f) || !isfinite(fx) || !isfinite(fy)) return all;
    float R[3][3], o[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[i][j] = c2w[4 * i + j];
        o[i] = c2w[4 * i + 3];
    }
    float A[3][3];  // adjugate: R^-1 = A / det
    A[0][0] = R[1][1] * R[2][2] - R[1][2] * R[2][1];
    A[0][1] = R[0][2] * R[2][1] - R[0][1] * R[2][2];
    A[0][2] = R[0][1] * R[1][2] - R[0][2] * R[1][1];
    A[1][0] = R[1][2] * R[2][0] - R[1][0] * R[2][2];
    A[1][1] = R[0][0] * R[2][2] - R[0][2] * R[2][0];
    A[1][2] = R[0][2] * R[1][0] - R[0][0] * R[1][2];
    A[2][0] = R[1][0] * R[2][1] - R[1][1] * R[2][0];
    A[2][1] = R[0][1] * R[2][0] - R[0][0] * R[2][1];
    A[2][2] = R[0][0] * R[1][1] - R[0][1] * R[1][0];
    const float det = R[0][0] * A[0][0] + R[0][1] * A[1][0] + R[0][2] * A[2][0];
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return all;
    const float idet = 1.f / det;
    float P[8][3];
    for (int c = 0; c < 8; ++c) {
        const float w[3] = {(c & 1) ? bh[0] : bl[0], (c & 2) ? bh[1] : bl[1], (c & 4) ? bh[2] : bl[2]};
        for (int i = 0; i < 3; ++i)
            P[c][i] = (A[i][0] * (w[0] - o[0]) + A[i][1] * (w[1] - o[1]) + A[i][2] * (w[2] - o[2])) * idet;
    }
    float zc;
    if (t0 > 0.f) {
        const float mx = fmaxf(fabsf(0.5f - cx), fabsf(W - 0.5f - cx)) / fabsf(fx);
        const float my = fmaxf(fabsf(0.5f - cy), fabsf(H - 0.5f - cy)) / fabsf(fy);
        zc = 0.5f * t0 / sqrtf(1.f + mx * mx + my * my);
    } else {
        for (int c = 0; c < 8; ++c)
            if (!(P[c][2] > 0.f)) return all;
        zc = 0.f;
    }
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    bool any = false;
    auto add = [&](float X, float Y, float Z) {
        const float iz = 1.f / Z;
        const float u = fx * X * iz + cx - 0.5f, v = fy * Y * iz + cy - 0.5f;
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
        any = true;
    };
    for (int c = 0; c < 8; ++c)
        if (P[c][2] >= zc && P[c][2] > 0.f) add(P[c][0], P[c][1], P[c][2]);
    if (zc > 0.f)
        for (int c = 0; c < 8; ++c)
            for (int b = 1; b < 8; b <<= 1) {
                if (c & b) continue;
                const float za = P[c][2], zb = P[c | b][2];
                if ((za < zc) == (zb < zc)) continue;
                const float s = (zc - za) / (zb - za);
                add(P[c][0] + s * (P[c | b][0] - P[c][0]), P[c][1] + s * (P[c | b][1] - P[c][1]), zc);
            }
    if (!any || !(umin <= umax) || !(vmin <= vmax)) return none;
    const float u0 = fmaxf(floorf(umin) - 2.f, 0.f), u1 = fminf(ceilf(umax) + 2.f, W - 1.f);
    const float v0 = fmaxf(floorf(vmin) - 2.f, 0.f), v1 = fminf(ceilf(vmax) + 2.f, H - 1.f);
    if (!(u0 <= u1) || !(v0 <= v1)) return none;
    return make_int4((int)u0, (int)v0, (int)u1, (int)v1);
}

// Morton cell of the centre of the voxel box [lo, hi]: per axis the centre voxel
// scaled to pm_cell_bits(axis) bits, the bits interleaved (x lowest).
__device__ __forceinline__ int morton_cell(const int lo[3], const int hi[3], const int n[3]) {
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long mid = ((long long)lo[a] + hi[a]) >> 1;
        c[a] = (int)min((long long)(1 << pm_cell_bits(a)) - 1, (mid << pm_cell_bits(a)) / max(n[a], 1));
    }
    int key = 0, bit = 0;
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (b < pm_cell_bits(a)) key |= ((c[a] >> b) & 1) << bit++;
    return key;
}
static_assert(pm_cell_bits(0) + pm_cell_bits(1) + pm_cell_bits(2) == 12 && PM_CELLS == 4096, "cell key width");
static_assert(NRAW + SQ_MAX_CLASSES <= PM_VISIT_SLOT, "the visit count needs a free slot of the tile row");

// One warp per primitive of the batch, a lane per camera: the rectangle in
// every camera, the number of candidate pixels and the box's Morton cell.
__global__ void k_pm_rects(Batch B, PmArgs A) {
    const int g = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (g >= A.ntot) return;
    const int s = scene_of_prim(A.poff, B.n, g);
    const SceneDesc& S = B.d[s];
    const int k = g - (int)__ldg(A.poff + s);
    const int4 b = __ldg(S.boxes + k);
    const int lo[3] = {b.x & 0xffff, b.y & 0xffff, b.z & 0xffff};
    const int hi[3] = {(int)((unsigned)b.x >> 16), (int)((unsigned)b.y >> 16), (int)((unsigned)b.z >> 16)};
    const bool ok = *S.status == SQ_OK && *S.save_status == SQ_OK && lo[0] <= hi[0] && lo[1] <= hi[1] &&
                    lo[2] <= hi[2];
    float bl[3], bh[3];
    for (int a = 0; a < 3; ++a) {
        bl[a] = S.g.lo[a] + (float)lo[a] * S.g.vs[a];
        bh[a] = S.g.lo[a] + (float)(hi[a] + 1) * S.g.vs[a];
    }
    const bool rays = S.n_cam > 0 && S.H > 0 && S.W > 0;  // t may be NULL without rays
    const float t0 = rays ? __ldg(S.t) : 0.f;
    int4* rect = S.pm_rect + (size_t)k * S.n_cam;
    long long total = 0;
    for (int c = lane; c < (rays ? S.n_cam : 0); c += 32) {
        const int4 rc = ok ? box_rect(S.K + 4 * c, S.c2w + 12 * c, S.H, S.W, bl, bh, t0) : make_int4(0, 0, -1, -1);
        rect[c] = rc;
        if (rc.z >= rc.x && rc.w >= rc.y) total += (long long)(rc.z - rc.x + 1) * (rc.w - rc.y + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) {
        A.cnt[g] = (int)total;  // at most the scene's ray count (< 2^31)
        A.key[g] = ok ? morton_cell(lo, hi, S.g.n) : 0;
    }
}

// Exclusive scan of the tile counts over all primitives (one block).
__global__ void __launch_bounds__(1024) k_pm_scan(PmArgs A) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (A.ntot + 1023) / 1024;
    const int b = min(A.ntot, tid * per), e = min(A.ntot, b + per);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += tiles_of(A.cnt[i]);
    const int incl = warp_incl_scan(sum, lane);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = wsum[lane];
        const int wi = warp_incl_scan(w, lane);
        wsum[lane] = wi - w;
    }
    __syncthreads();
    int run = wsum[wid] + incl - sum;
    for (int i = b; i < e; ++i) {
        A.toff[i] = run;
        const int nt = tiles_of(A.cnt[i]);
        for (int t = 0; t < nt; ++t) A.tprim[run + t] = i;
        run += nt;
    }
    if (tid == 1023) A.toff[A.ntot] = run;
    __syncthreads();

    // The queue: per scene, the primitives' tiles bucketed by Morton cell (a
    // counting sort in shared memory); within a cell the order the shared-memory
    // atomics give, which moves only the schedule, never a sum.
    __shared__ int hist[PM_CELLS];
    int qbase = 0;
    for (int s = 0; s < A.nscene; ++s) {
        const int p0 = (int)A.poff[s], p1 = (int)A.poff[s + 1];
        for (int c = tid; c < PM_CELLS; c += 1024) hist[c] = 0;
        __syncthreads();
        for (int i = p0 + tid; i < p1; i += 1024) {
            const int nt = A.toff[i + 1] - A.toff[i];
            if (nt > 0) atomicAdd(&hist[A.key[i]], nt);
        }
        __syncthreads();
        constexpr int PER = PM_CELLS / 1024;
        int loc[PER], lsum = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            loc[i] = hist[tid * PER + i];
            lsum += loc[i];
        }
        const int li = warp_incl_scan(lsum, lane);
        if (lane == 31) wsum[wid] = li;
        __syncthreads();
        if (wid == 0) {
            const int w = wsum[lane];
            wsum[lane] = warp_incl_scan(w, lane) - w;
        }
        __syncthreads();
        int at = qbase + wsum[wid] + li - lsum;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            hist[tid * PER + i] = at;
            at += loc[i];
        }
        const int scene_tiles = A.toff[p1] - A.toff[p0];
        __syncthreads();
        for (int i = p0 + tid; i < p1; i += 1024) {
            const int t0 = A.toff[i], nt = A.toff[i + 1] - t0;
            if (nt <= 0) continue;
            const int q = atomicAdd(&hist[A.key[i]], nt);
            for (int t = 0; t < nt; ++t) A.qtile[q + t] = t0 + t;
        }
        qbase += scene_tiles;
        __syncthreads();
    }
}

// Ray direction of every ray of the batch (pixel_ray) and its number of
// composited samples (in .w), for the candidate pixels of the tiles: one thread
// per ray.
__global__ void k_pm_dirs(Batch B) {
    const long long gr = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gr >= B.total) return;
    const int s = scene_of(B, gr);
    const SceneDesc& S = B.d[s];
    const long long r = gr - __ldg(B.off + s);
    float o[3], d[3];
    scene_ray(S, r, o, d);
    const int Le = min(max(__ldg(S.save_n + r), 0), S.L);
    S.pm_dir[r] = make_float4(d[0], d[1], d[2], __int_as_float(Le));
}

// grad_sem of every ray of the batch copied to rows of CP classes (zero padding),
// so that a tile reads a ray's row with CP / 4 aligned vector loads: one thread
// per (ray, group of four classes), threadIdx.x the group, threadIdx.y the ray.
__global__ void k_pm_gs(Batch B) {
    const long long gr = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (gr >= B.total) return;
    const int cp4 = B.d[0].cp >> 2;  // the scenes of a batch share n_classes
    const int q = (int)threadIdx.x;
    const int s = scene_of(B, gr);
    const SceneDesc& S = B.d[s];
    const long long r = gr - __ldg(B.off + s);
    const float* row = S.grad_sem + r * S.C;
    float v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = 4 * q + c < S.C ? __ldg(row + 4 * q + c) : 0.f;
    S.pm_gs[r * cp4 + q] = make_float4(v[0], v[1], v[2], v[3]);
}

// Scaled coordinate of sample j on one axis, rounded as sample_voxel rounds it,
// tested against a threshold: (u_j < thr) != neg.
__device__ __forceinline__ bool below(const float* ts, int j, float o, float d, float glo, float inv, float thr,
                                      bool neg) {
    const float x = __fadd_rn(o, __fmul_rn(ts[j], d));
    const float u = __fmul_rn(__fsub_rn(x, glo), inv);
    return (u < thr) != neg;
}

// Number of leading samples j of [0, Le) with below(j).  u_j is monotone in j (t
// non-decreasing), so the predicate holds on a prefix: a binary search finds its
// length.
__device__ __noinline__ int lead_search(const float* ts, int Le, float o, float d, float glo, float inv, float thr,
                                        bool neg) {
    int n = 0;
    for (int step = Le > 0 ? 1 << (31 - __clz(Le)) : 0; step > 0; step >>= 1)
        if (n + step <= Le && below(ts, n + step - 1, o, d, glo, inv, thr, neg)) n += step;
    return n;
}

// Estimated prefix length: the ray meets the plane u = thr at t* = (lo + thr vs -
// o) / d (id: an approximate 1 / d), and with evenly spaced samples about
// (t* - t_0) / dt samples lie before it.
__device__ __forceinline__ int lead_est(float o, float id, float glo, float vs, float thr, float t0, float inv_dt,
                                        int Le) {
    const float tstar = (fmaf(thr, vs, glo) - o) * id;
    const float fe = ceilf((tstar - t0) * inv_dt);
    return (int)fminf(fmaxf(fe, 0.f), (float)Le);
}

// The same prefix length, starting from an estimate n (lead_est), which is moved
// to the exact boundary by testing the predicate itself (at most a few steps each
// way, then the binary search), so the result never depends on the estimate's
// rounding; exact for any n in [0, Le], a ray parallel to the axis included.
__device__ __forceinline__ int lead_at(const float* ts, int Le, float o, float d, float glo, float inv, float thr,
                                       bool neg, int n) {
    for (int k = 0; n > 0 && !below(ts, n - 1, o, d, glo, inv, thr, neg); ++k) {
        if (k == 4) return lead_search(ts, Le, o, d, glo, inv, thr, neg);
        --n;
    }
    for (int k = 0; n < Le && below(ts, n, o, d, glo, inv, thr, neg); ++k) {
        if (k == 4) return lead_search(ts, Le, o, d, glo, inv, thr, neg);
        ++n;
    }
    return n;
}

// Sample j's voxel (the forward's FP32 rule) inside the box [blo, bhi) on every axis.
__device__ __forceinline__ bool in_box(const float* ts, int j, const float o[3], const float d[3], const GridC& g,
                                       const float blo[3], const float bhi[3]) {
    const float tj = ts[j];
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = __fmul_rn(__fsub_rn(__fadd_rn(o[a], __fmul_rn(tj, d[a])), g.lo[a]), g.inv_vs[a]);
        in = in && u >= blo[a] && u < bhi[a];
    }
    return in;
}

struct PmSmem {
    // the pass's non-empty runs in candidate order, run e at index e
    float d[3][PM_CHUNK];        // ray direction
    float cd[PM_CHUNK];          // <dL/dS of the ray, c_k>
    int r[PM_CHUNK];             // ray index in its scene
    int jc[PM_CHUNK];            // first sample of the run | camera << 10
    int pre[PM_CHUNK + 1];       // exclusive prefix of the run lengths (pairs); the pass's pairs from nnz on
    float wsum[PM_CHUNK];        // sum over the run of w_j p_o
    float ts[SQ_MAX_SAMPLES];    // sample distances of the tile's scene
    int4 rc[PM_SMCAM];           // the primitive's rectangles (n_cam <= PM_SMCAM)
    int rpre[PM_SMCAM + 1];      // exclusive prefix of their pixel counts
    int head_slot[PM_THREADS];   // run a thread's slice starts inside (-1: none)
    float head_val[PM_THREADS];  // that thread's part of the run's w p_o sum
    float red[PM_WARPS][NRAW];
    float4 cacc[PM_WARPS][PM_CSUB][8];  // class gradient partials: per warp and run lane group, classes 4q..4q+3
    alignas(16) float lp[32];    // class vector of the tile's primitive (lpad row)
    int wtot[PM_WARPS];
    int ztot[PM_WARPS];
    int tile;
};
static_assert(SQ_MAX_SAMPLES <= 1024, "first samples are packed in 10 bits");

__device__ __forceinline__ void camera_origin(const SceneDesc& S, int cam, float o[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = __ldg(S.c2w + 12 * cam + 4 * a + 3);
}

template <int CP>
__global__ void __launch_bounds__(PM_THREADS, 4) k_pm_tiles(Batch B, PmArgs A) {
    __shared__ PmSmem sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ntiles = __ldg(A.toff + A.ntot);
    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(A.ctr, 1);
            sh.tile = q < ntiles ? __ldg(A.qtile + q) : -1;
        }
        __syncthreads();
        const int tile = sh.tile;
        if (tile < 0) break;
        const int g = __ldg(A.tprim + tile);
        const int s = scene_of_prim(A.poff, B.n, g);
        const SceneDesc& S = B.d[s];
        const int k = g - (int)__ldg(A.poff + s);
        const int it = tile - __ldg(A.toff + g), nt = __ldg(A.toff + g + 1) - __ldg(A.toff + g);
        const long long nc = __ldg(A.cnt + g);
        const int cbeg = (int)(nc * it / nt), cend = (int)(nc * (it + 1) / nt);
        const int L = S.L, C = S.C, H = S.H, W = S.W, ncam = S.n_cam;
        const BwdPrim P = load_bwd(S.rec, S.aux, k);
        const int4 bx = __ldg(S.boxes + k);
        const float blo[3] = {(float)(bx.x & 0xffff), (float)(bx.y & 0xffff), (float)(bx.z & 0xffff)};
        const float bhi[3] = {(float)(((unsigned)bx.x >> 16) + 1u), (float)(((unsigned)bx.y >> 16) + 1u),
                              (float)(((unsigned)bx.z >> 16) + 1u)};
        const int4* __restrict__ rect = S.pm_rect + (size_t)k * ncam;
        if (tid < CP) sh.lp[tid] = __ldg(S.lpad + (size_t)k * CP + tid);
        for (int j = tid; j < L; j += PM_THREADS) sh.ts[j] = __ldg(S.t + j);
        const bool rc_sm = ncam <= PM_SMCAM;
        if (rc_sm && tid < 32) {  // rectangles and the prefix of their pixel counts
            int area = 0;
            if (tid < ncam) {
                const int4 rc = __ldg(rect + tid);
                const int w = rc.z - rc.x + 1, h = rc.w - rc.y + 1;
                area = (w > 0 && h > 0) ? w * h : 0;
                sh.rc[tid] = rc;
            }
            const int incl = warp_incl_scan(area, lane);
            if (tid <= ncam) sh.rpre[tid] = incl - area;
        }
        float bwl[3], bwh[3];  // world extent of the box (for the slab test)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bwl[a] = fmaf(blo[a], S.g.vs[a], S.g.lo[a]);
            bwh[a] = fmaf(bhi[a], S.g.vs[a], S.g.lo[a]);
        }
        const float t0 = __ldg(S.t), tl = __ldg(S.t + L - 1);
        const float inv_dt = (L > 1 && tl > t0) ? (float)(L - 1) / (tl - t0) : 0.f;
        float acc[13];
#pragma unroll
        for (int i = 0; i < 13; ++i) acc[i] = 0.f;
        int tpairs = 0;  // pairs of the tile (the same value in every thread)
        for (int i = tid; i < PM_WARPS * PM_CSUB * 8; i += PM_THREADS)
            (&sh.cacc[0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();

        for (int cb = cbeg; cb < cend; cb += PM_CHUNK) {
            // ---- candidates -> runs: thread tid holds candidates cb + tid * PM_CPT + i.
            // Three stages over the thread's candidates, so that the loads of all of
            // them are in flight together.
            int rr[PM_CPT], cam[PM_CPT], Le[PM_CPT], j0s[PM_CPT], len[PM_CPT];
            float4 dv[PM_CPT];
#pragma unroll
            for (int i = 0; i < PM_CPT; ++i) {  // pixel of the candidate
                const int ci = cb + tid * PM_CPT + i;
                rr[i] = -1;
                cam[i] = 0;
                if (ci >= cend) continue;
                int c = 0, rem = ci;
                int4 rc = make_int4(0, 0, -1, -1);
                if (rc_sm) {
                    while (c < ncam && sh.rpre[c + 1] <= ci) ++c;
                    if (c >= ncam) continue;
                    rc = sh.rc[c];
                    rem = ci - sh.rpre[c];
                } else {
                    for (; c < ncam; ++c) {
                        rc = __ldg(rect + c);
                        const int w = rc.z - rc.x + 1, h = rc.w - rc.y + 1;
                        const int area = (w > 0 && h > 0) ? w * h : 0;
                        if (rem < area) break;
                        rem -= area;
                    }
                    if (c >= ncam) continue;
                }
                const int w = rc.z - rc.x + 1;
                rr[i] = (c * H + rc.y + rem / w) * W + rc.x + rem % w;
                cam[i] = c;
            }
#pragma unroll
            for (int i = 0; i < PM_CPT; ++i) {  // its ray direction and composited samples
                dv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                Le[i] = 0;
                if (rr[i] >= 0) {
                    dv[i] = __ldg(S.pm_dir + rr[i]);
                    Le[i] = __float_as_int(dv[i].w);
                }
            }
            int tl_sum = 0;
#pragma unroll
            for (int i = 0; i < PM_CPT; ++i) {  // the run: samples of the ray inside the box
                len[i] = 0;
                j0s[i] = 0;
                if (Le[i] == 0) continue;
                const float d[3] = {dv[i].x, dv[i].y, dv[i].z};
                float o[3];
                camera_origin(S, cam[i], o);
                // Slab test of the segment t in [t_0, t_last] against the box grown by
                // dl, a bound (with a wide safety factor) on how far outside the box an
                // FP32 sample can be and still pass the FP32 voxel test: a miss here
                // means no composited sample of the ray lies in the box.
                const float tlast = sh.ts[Le[i] - 1];
                const float tm = fmaxf(fabsf(t0), fabsf(tlast));
                float te = t0, tx = tlast, id[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float dl = 1e-5f * (fabsf(o[a]) + fabsf(S.g.lo[a]) + fabsf(bwl[a]) + fabsf(bwh[a]) +
                                              tm * fabsf(d[a])) + 1e-6f;
                    if (fabsf(d[a]) < 1e-20f) {  // the ray keeps this coordinate
                        id[a] = 0.f;
                        if (o[a] < bwl[a] - dl || o[a] > bwh[a] + dl) te = INFINITY;
                    } else {
                        id[a] = rcp(d[a]);
                        const float t1 = (bwl[a] - dl - o[a]) * id[a], t2 = (bwh[a] + dl - o[a]) * id[a];
                        const float lo_t = fminf(t1, t2), hi_t = fmaxf(t1, t2);
                        te = fmaxf(te, lo_t - (1e-5f * fabsf(lo_t) + 1e-6f));
                        tx = fminf(tx, hi_t + (1e-5f * fabsf(hi_t) + 1e-6f));
                    }
                }
                if (!(te <= tx)) continue;
                // The samples inside the box form one interval (u_j is monotone in j on
                // every axis), so an interval whose end samples pass the voxel rule and
                // whose outer neighbours fail it is the exact one: the plane-crossing
                // estimates almost always give it, and the per-axis searches, started
                // from the same estimates, run only when the check fails (a sample
                // within rounding of a plane, a ray parallel to an axis, an empty
                // estimate).
                int j0 = 0, j1 = Le[i];
                bool fast = false;
                int ne[3], nx[3];  // estimated leads of the entry and exit planes
                int j0e = 0, j1e = Le[i];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const bool neg = d[a] < 0.f;
                    ne[a] = lead_est(o[a], id[a], S.g.lo[a], S.g.vs[a], neg ? bhi[a] : blo[a], t0, inv_dt, Le[i]);
                    nx[a] = lead_est(o[a], id[a], S.g.lo[a], S.g.vs[a], neg ? blo[a] : bhi[a], t0, inv_dt, Le[i]);
                    j0e = max(j0e, ne[a]);
                    j1e = min(j1e, nx[a]);
                }
                if (id[0] != 0.f && id[1] != 0.f && id[2] != 0.f) {
                    if (j0e < j1e && in_box(sh.ts, j0e, o, d, S.g, blo, bhi) &&
                        in_box(sh.ts, j1e - 1, o, d, S.g, blo, bhi) &&
                        (j0e == 0 || !in_box(sh.ts, j0e - 1, o, d, S.g, blo, bhi)) &&
                        (j1e == Le[i] || !in_box(sh.ts, j1e, o, d, S.g, blo, bhi))) {
                        j0 = j0e;
                        j1 = j1e;
                        fast = true;
                    }
                }
                if (!fast) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const bool neg = d[a] < 0.f;
                        j0 = max(j0, lead_at(sh.ts, Le[i], o[a], d[a], S.g.lo[a], S.g.inv_vs[a], neg ? bhi[a] : blo[a],
                                             neg, ne[a]));
                    }
                    if (j0 >= j1) continue;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const bool neg = d[a] < 0.f;
                        j1 = min(j1, lead_at(sh.ts, Le[i], o[a], d[a], S.g.lo[a], S.g.inv_vs[a], neg ? blo[a] : bhi[a],
                                             neg, nx[a]));
                    }
                    if (j1 <= j0) continue;
                }
                len[i] = j1 - j0;
                j0s[i] = j0;
                tl_sum += len[i];
            }
            // ---- exclusive scans, in candidate order, of the run lengths and of the
            // non-empty runs: the runs' data go to shared memory at their index, so the
            // walk and the class stages take runs e = 0 .. nnz - 1 with no empty slots
            int npairs, nnz;
            {
                int nzt = 0;
#pragma unroll
                for (int i = 0; i < PM_CPT; ++i) nzt += len[i] > 0 ? 1 : 0;
                const int il = warp_incl_scan(tl_sum, lane);
                const int zl = warp_incl_scan(nzt, lane);
                if (lane == 31) {
                    sh.wtot[wid] = il;
                    sh.ztot[wid] = zl;
                }
                __syncthreads();
                int wl = 0, tl2 = 0, zw = 0;
                nnz = 0;
#pragma unroll
                for (int w2 = 0; w2 < PM_WARPS; ++w2) {
                    const int a = sh.wtot[w2], z = sh.ztot[w2];
                    if (w2 < wid) {
                        wl += a;
                        zw += z;
                    }
                    tl2 += a;
                    nnz += z;
                }
                int pl = wl + il - tl_sum, zp = zw + zl - nzt;
#pragma unroll
                for (int i = 0; i < PM_CPT; ++i) {  // the non-empty runs' data at their index
                    if (len[i] == 0) continue;
                    sh.d[0][zp] = dv[i].x;
                    sh.d[1][zp] = dv[i].y;
                    sh.d[2][zp] = dv[i].z;
                    sh.r[zp] = rr[i];
                    sh.jc[zp] = j0s[i] | (cam[i] << 10);
                    sh.pre[zp] = pl;
                    pl += len[i];
                    ++zp;
                }
                npairs = tl2;
                tpairs += tl2;
                for (int e = nnz + tid; e <= PM_CHUNK; e += PM_THREADS) sh.pre[e] = tl2;  // bounds the run search
                sh.head_slot[tid] = -1;
            }
            __syncthreads();
            // ---- <dL/dS of the ray, c_k> of each non-empty run: lane (sub, q) of a warp
            // reads float4 q of run sub's padded gS row (a row is 8 lanes' contiguous
            // loads), two runs per lane group in flight; the group sums its lanes'
            // partial dot products in a fixed tree
            {
                const int sub = lane >> 3, q = lane & 7;
                const unsigned gm = 0xffu << (lane & 24);
                const float4 l4 = q < CP / 4 ? reinterpret_cast<const float4*>(sh.lp)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                constexpr int STEP = PM_WARPS * PM_CSUB;
                for (int e = wid * PM_CSUB + sub; e < nnz; e += 2 * STEP) {
                    const int e2 = e + STEP;
                    const int s1 = e, s2 = e2 < nnz ? e2 : -1;
                    float4 g1 = make_float4(0.f, 0.f, 0.f, 0.f), g2 = g1;
                    if (q < CP / 4) {
                        g1 = __ldg(S.pm_gs + (long long)sh.r[s1] * (CP / 4) + q);
                        if (s2 >= 0) g2 = __ldg(S.pm_gs + (long long)sh.r[s2] * (CP / 4) + q);
                    }
                    float v1 = fmaf(g1.w, l4.w, fmaf(g1.z, l4.z, fmaf(g1.y, l4.y, g1.x * l4.x)));
                    float v2 = fmaf(g2.w, l4.w, fmaf(g2.z, l4.z, fmaf(g2.y, l4.y, g2.x * l4.x)));
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        v1 += __shfl_xor_sync(gm, v1, o);
                        v2 += __shfl_xor_sync(gm, v2, o);
                    }
                    if (q == 0) {
                        sh.cd[s1] = v1;
                        if (s2 >= 0) sh.cd[s2] = v2;
                    }
                }
            }
            __syncthreads();

            // ---- walk: thread tid takes pairs [p, p1), the slices in thread order
            // (empty slices only at the end).  Each step evaluates up to PM_NS pairs of
            // one run; the next step's (dL/dalpha_j, w_j) loads are issued before
            // this step's arithmetic (the gathers are latency-bound).
            {
                const int q = npairs / PM_THREADS, rm = npairs % PM_THREADS;
                int p = tid * q + min(tid, rm);
                const int p1 = p + q + (tid < rm ? 1 : 0);
                if (p < p1) {
                    int slot = 0;
#pragma unroll
                    for (int step = PM_CHUNK / 2; step > 0; step >>= 1)
                        if (sh.pre[slot + step] <= p) slot += step;
                    bool head = sh.pre[slot] < p;
                    float o[3], d[3];
                    int jcs = sh.jc[slot];
                    camera_origin(S, jcs >> 10, o);
#pragma unroll
                    for (int a = 0; a < 3; ++a) d[a] = sh.d[a][slot];
                    float cd = sh.cd[slot];
                    const float2* gwr = S.gw + (long long)sh.r[slot] * L;
                    int jj = (jcs & 1023) + (p - sh.pre[slot]);
                    int rend = sh.pre[slot + 1];
                    int se = min(rend, p1);
                    int m = min(PM_NS, se - p);  // pairs of this step
                    float2 gq[PM_NS];
#pragma unroll
                    for (int i = 0; i < PM_NS; ++i) gq[i] = i < m ? gwr[jj + i] : make_float2(0.f, 0.f);
                    for (;;) {
                        const int pn = p + m;
                        // the next step: same run, or the next run (its data read every
                        // step, selected without a branch); its loads are issued before
                        // this step's arithmetic
                        const bool more = pn < p1;
                        const bool sw = more && pn == rend;
                        const int slot_n = slot + (sw ? 1 : 0);
                        const int jcn = sh.jc[slot_n], rn = sh.r[slot_n], pren = sh.pre[slot_n + 1];
                        const int jj_n = sw ? (jcn & 1023) : jj + m, rend_n = sw ? pren : rend;
                        const float2* gwr_n = sw ? S.gw + (long long)rn * L : gwr;
                        const int se_n = min(rend_n, p1);
                        const int m_n = more ? min(PM_NS, se_n - pn) : 0;
                        float2 gq_n[PM_NS];
#pragma unroll
                        for (int i = 0; i < PM_NS; ++i)
                            gq_n[i] = i < m_n ? gwr_n[jj_n + i] : make_float2(0.f, 0.f);
                        // this step's pairs
#pragma unroll
                        for (int i = 0; i < PM_NS; ++i) {
                            if (i < m) {
                                const float tj = sh.ts[jj + i];
                                float x[3], pr[11];
#pragma unroll
                                for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(tj, d[a]));
                                const float po = occupancy_partials(P, x, pr);
                                if (po != 0.f) accumulate(acc, po, pr, gq[i].x, gq[i].y, P.f.sigma, cd);
                            }
                        }
                        if (pn == se) {  // the run's part in this slice is done
                            if (head) {
                                sh.head_slot[tid] = slot;
                                sh.head_val[tid] = acc[12];
                                head = false;
                            } else {
                                sh.wsum[slot] = acc[12];
                            }
                            acc[12] = 0.f;
                        }
                        if (!more) break;
                        jcs = sh.jc[slot_n];
                        camera_origin(S, jcs >> 10, o);
#pragma unroll
                        for (int a = 0; a < 3; ++a) d[a] = sh.d[a][slot_n];
                        cd = sh.cd[slot_n];
                        slot = slot_n;
                        jj = jj_n;
                        rend = rend_n;
                        gwr = gwr_n;
                        se = se_n;
                        m = m_n;
#pragma unroll
                        for (int i = 0; i < PM_NS; ++i) gq[i] = gq_n[i];
                        p = pn;
                    }
                }
            }
            __syncthreads();
            // ---- runs shared by several slices: the owner's part, then the others' in thread order
            {
                const int hs = sh.head_slot[tid];
                if (hs >= 0 && (tid == 0 || sh.head_slot[tid - 1] != hs)) {
                    float v = sh.wsum[hs];
                    for (int t2 = tid; t2 < PM_THREADS && sh.head_slot[t2] == hs; ++t2) v += sh.head_val[t2];
                    sh.wsum[hs] = v;
                }
            }
            __syncthreads();
            // ---- class gradient of the runs, sum over runs of (sum_j w_j p_o) dL/dS_ray:
            // the non-empty runs in list order, PM_CSUB per warp at a time; lane
            // (sub, q) reads classes 4q..4q+3 of run sub's padded gS row and keeps
            // their partial sums in its warp's accumulator row (fixed order)
            {
                const int sub = lane >> 3, q = lane & 7;
                if (q < CP / 4) {
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int e = wid * PM_CSUB + sub; e < nnz; e += PM_WARPS * PM_CSUB) {
                        const float wv = sh.wsum[e];
                        const float4 g4 = __ldg(S.pm_gs + (long long)sh.r[e] * (CP / 4) + q);
                        a.x = fmaf(wv, g4.x, a.x);
                        a.y = fmaf(wv, g4.y, a.y);
                        a.z = fmaf(wv, g4.z, a.z);
                        a.w = fmaf(wv, g4.w, a.w);
                    }
                    float4& c4 = sh.cacc[wid][sub][q];
                    c4 = make_float4(c4.x + a.x, c4.y + a.y, c4.z + a.z, c4.w + a.w);
                }
                __syncthreads();
            }
        }
        // ---- the tile's sums
#pragma unroll
        for (int i = 0; i < NRAW; ++i) {
            const float v = warp_sum(acc[i]);
            if (lane == 0) sh.red[wid][i] = v;
        }
        __syncthreads();
        float* out = A.part + (size_t)tile * GF;
        if (tid < NRAW) {
            float v = 0.f;
#pragma unroll
            for (int w2 = 0; w2 < PM_WARPS; ++w2) v += sh.red[w2][tid];
            out[tid] = v;
        }
        if (tid < C) {  // the warps' and lane groups' class partials in a fixed order
            float cg = 0.f;
            for (int w2 = 0; w2 < PM_WARPS; ++w2)
#pragma unroll
                for (int s2 = 0; s2 < PM_CSUB; ++s2) cg += (&sh.cacc[w2][s2][0].x)[tid];
            out[NRAW + tid] = cg;
        }
        if (tid == 0) out[PM_VISIT_SLOT] = __int_as_float(tpairs);
        __syncthreads();
    }
}

// Each primitive's accumulator row: its tiles' sums in tile order.
__global__ void k_pm_final(Batch B, PmArgs A) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = (int)(idx / GF), i = (int)(idx % GF);
    if (g >= A.ntot) return;
    const int s = scene_of_prim(A.poff, B.n, g);
    const SceneDesc& S = B.d[s];
    const int k = g - (int)__ldg(A.poff + s);
    if (i == PM_VISIT_SLOT) {  // pairs the tiles of the primitive evaluated
        if (S.pair_visits) {
            long long nv = 0;
            const int t0 = __ldg(A.toff + g), t1 = __ldg(A.toff + g + 1);
#pragma unroll 4
            for (int t = t0; t < t1; ++t) nv += __float_as_int(__ldg(A.part + (size_t)t * GF + i));
            S.pair_visits[k] = nv;
        }
        return;
    }
    if (i >= NRAW + S.C) return;
    float v = 0.f;  // in tile order
    const int t0 = __ldg(A.toff + g), t1 = __ldg(A.toff + g + 1);
#pragma unroll 4
    for (int t = t0; t < t1; ++t) v += __ldg(A.part + (size_t)t * GF + i);
    S.gacc[(size_t)k * GF + i] = v;
}

}  // namespace

sq_status_t launch_backward_pm(const Batch& B, const PmArgs& A, int cp, cudaStream_t st) {
    if (A.ntot == 0) return SQ_OK;
    const void* fn = nullptr;
    switch (cp) {
        case 4: fn = (const void*)k_pm_tiles<4>; break;
        case 8: fn = (const void*)k_pm_tiles<8>; break;
        case 12: fn = (const void*)k_pm_tiles<12>; break;
        case 16: fn = (const void*)k_pm_tiles<16>; break;
        case 20: fn = (const void*)k_pm_tiles<20>; break;
        case 24: fn = (const void*)k_pm_tiles<24>; break;
        case 28: fn = (const void*)k_pm_tiles<28>; break;
        case 32: fn = (const void*)k_pm_tiles<32>; break;
        default:
            set_last_error("n_classes padding %d not supported", cp);
            return SQ_ERR_INVALID_ARG;
    }
    SQ_LAUNCH("k_pm_rects", st, k_pm_rects<<<(unsigned)(((long long)A.ntot * 32 + 127) / 128), 128, 0, st>>>(B, A));
    if (B.total > 0) {
        SQ_LAUNCH("k_pm_dirs", st, k_pm_dirs<<<(unsigned)((B.total + 255) / 256), 256, 0, st>>>(B));
        SQ_LAUNCH("k_pm_gs", st, k_pm_gs<<<(unsigned)((B.total + 63) / 64), dim3(cp / 4, 64), 0, st>>>(B));
    }
    SQ_LAUNCH("k_pm_scan", st, k_pm_scan<<<1, 1024, 0, st>>>(A));
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PM_THREADS, 0);
    if (e != cudaSuccess) return cuda_status(e, "k_pm_tiles occupancy");
    long long blocks = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    const long long most = (long long)A.ntot * PM_MAXT;
    if (blocks > most) blocks = most;
    Batch barg = B;
    PmArgs aarg = A;
    void* args[] = {&barg, &aarg};
    prof_begin("k_pm_tiles", st);
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(PM_THREADS), args, 0, st);
    prof_end(st);
    if (e != cudaSuccess) return cuda_status(e, "k_pm_tiles");
    const long long nf = (long long)A.ntot * GF;
    SQ_LAUNCH("k_pm_final", st, k_pm_final<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(B, A));
    return SQ_OK;
}

}  // namespace sqr
