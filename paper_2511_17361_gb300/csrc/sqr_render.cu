// sqr_render.cu -- forward and backward superquadric volume rendering (Sec. 3.3.2,
// 3.3.3) on sm_103a.
//
// Forward (and the replay phase of the backward): a warp marches four rays at a
// time, eight lanes per ray, one lane per sample.  Each lane walks its own voxel
// list (Sec. 3.3.1), so the sums of Eq. 4 (alpha = sum p sigma, s = sum p c) stay
// in the lane's registers; compositing (Eq. 5-6) of the eight samples is an
// 8-lane product scan of (1 - alpha).  Rays are handed out by a global counter,
// so a lane group whose ray ends early takes the next ray.
//
// Backward gradients: one warp per ray.  Along a ray the samples that list a
// given primitive are contiguous (a ray crosses a primitive's voxel box once), so
// every primitive of the current sample's list is given an owner slot in a lane;
// the owner accumulates that primitive's parameter gradients in registers for as
// long as it stays in the lists and flushes them once when it leaves, as one
// coalesced 32-wide atomic add into a [N, 32] accumulator.  The replay that
// precedes it keeps per sample alpha_j, v_j = gD t_j + <gS, s_j> and T_j in shared
// memory; the back-to-front sweep U_j = alpha_{j+1} v_{j+1} + (1 - alpha_{j+1}) U_{j+1}
// then gives dL/dalpha_j = T_j (v_j - U_j) (zero where the clamp is active) and
// w_j = T_j alpha_j.
#include <limits.h>
#include <math.h>

#include "sqr_common.cuh"

namespace sqr {

namespace {

#ifndef SQR_MIGRATE
#define SQR_MIGRATE 0
#endif
constexpr int GS = 8;       // lanes (samples) per ray in the forward
constexpr int OWN = 64;     // owner slots per warp (two per lane)
constexpr int QCAP = 64;    // pending gradient flushes per warp (backward)
constexpr int QW = 16;      // words per pending flush: key, 12 geometry, sigma, W, pad
constexpr int GF = 48;      // floats per primitive in the gradient accumulator (13 + up to 32 classes)
constexpr int NGEO = 13;    // m3 q4 s3 eps2 sigma1
constexpr int NRAW = 12;    // summed partials: gx3 tau3 u.df/du 3 eps2 sigma1
constexpr int FWD_WARPS = 8;
constexpr int BWD_WARPS = 8;

// ------------------------------------------------------------------ packing
__global__ void k_pack(sq_prims_t P, float4* __restrict__ rec, float4* __restrict__ aux, float* __restrict__ lpad,
                       int cp) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n) return;
    float w = P.quats[4 * k + 0], x = P.quats[4 * k + 1], y = P.quats[4 * k + 2], z = P.quats[4 * k + 3];
    float nq = sqrtf(w * w + x * x + y * y + z * z);
    float inq = 1.0f / nq;
    w *= inq; x *= inq; y *= inq; z *= inq;
    float R[3][3];
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
    float is[3] = {1.f / P.scales[3 * k + 0], 1.f / P.scales[3 * k + 1], 1.f / P.scales[3 * k + 2]};
    float e1 = P.eps[2 * k + 0], e2 = P.eps[2 * k + 1];
    float ea = 2.f / e2, eb = e2 / e1, ec = 2.f / e1;
    float M[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) M[j][i] = R[i][j] * is[j];
    float4* r = rec + (size_t)k * REC4;
    r[0] = make_float4(P.means[3 * k + 0], P.means[3 * k + 1], P.means[3 * k + 2], P.opacity[k]);
    r[1] = make_float4(M[0][0], M[0][1], M[0][2], ea);
    r[2] = make_float4(M[1][0], M[1][1], M[1][2], eb);
    r[3] = make_float4(M[2][0], M[2][1], M[2][2], ec);
    if (aux) {
        float4* a = aux + (size_t)k * AUX4;
        a[0] = make_float4(w, x, y, z);
        a[1] = make_float4(inq, is[0], is[1], is[2]);
        a[2] = make_float4(e1, e2, 1.f / e1, 1.f / e2);
    }
    const int C = P.n_classes;
    for (int c = 0; c < cp; ++c) lpad[(size_t)k * cp + c] = c < C ? P.logits[(size_t)k * C + c] : 0.f;
}

// ------------------------------------------------------------------ shared args
struct RenderArgs {
    const float4* rec;
    const float4* aux;
    const float* lpad;  // [N, CP]
    const int* v_n;
    const int* v_f;
    const int* v_sq;
    const int* status;
    GridC g;
    const float* K;
    const float* c2w;
    const float* t;
    int n_cam, H, W, L, C;
    long long R;
    float kappa, alpha_max;
    int* ray_ctr;     // work counter, zeroed before the launch
    int4* boxes;      // packed voxel boxes (backward)
    float* save_T;    // [R, L] transmittance before each sample (forward writes, backward reads)
    int* save_n;      // [R] samples composited
};

__device__ __forceinline__ void ray_of(const RenderArgs& a, long long r, float o[3], float d[3]) {
    long long hw = (long long)a.H * a.W;
    int cam = (int)(r / hw);
    long long pix = r - (long long)cam * hw;
    int v = (int)(pix / a.W), u = (int)(pix - (long long)v * a.W);
    pixel_ray(a.K + 4 * cam, a.c2w + 12 * cam, u, v, o, d);
}

// Inclusive product scan within aligned groups of GS lanes.
__device__ __forceinline__ float group_incl_prod(float v, int s) {
#pragma unroll
    for (int o = 1; o < GS; o <<= 1) {
        float y = __shfl_up_sync(0xffffffffu, v, o, GS);
        if (s >= o) v *= y;
    }
    return v;
}

// Compositing (Eq. 5) of a group's GS consecutive samples.  Lane s holds alpha
// (0 for lanes past L or outside the grid).  Returns w = T_before * alpha (0 past
// an early termination) and T_before; advances T (uniform in the group); `stop`
// when kappa > 0 ends the ray inside this chunk, `used` = samples composited.
__device__ __forceinline__ float group_composite(float alpha, int s, int gbase, float kappa, float& T, float& Tb,
                                                 bool valid, int& used, bool& stop) {
    const float incl = group_incl_prod(1.f - alpha, s);
    float excl = __shfl_up_sync(0xffffffffu, incl, 1, GS);
    if (s == 0) excl = 1.f;
    Tb = T * excl;
    float w = Tb * alpha;
    used = GS;
    stop = false;
    const unsigned kill = __ballot_sync(0xffffffffu, valid && kappa > 0.f && T * incl < kappa);
    const unsigned gk = (kill >> gbase) & ((1u << GS) - 1u);
    if (gk) {
        const int ls = __ffs(gk) - 1;
        if (s > ls) w = 0.f;
        used = ls + 1;
        stop = true;
    }
    const float tot = __shfl_sync(0xffffffffu, incl, gbase + (gk ? (__ffs(gk) - 1) : GS - 1));
    T = T * tot;
    return w;
}

// ------------------------------------------------------------------ forward
// Four rays per warp, eight lanes per ray, one lane per sample: each lane walks
// its own voxel list with alpha and s_j in registers (Eq. 4), the group composites
// its eight samples with a product scan (Eq. 5-6), and saves T_j for the backward.
template <int CP>
__global__ void __launch_bounds__(FWD_WARPS * 32) k_forward(RenderArgs a, float* __restrict__ depth,
                                                            float* __restrict__ sem, float* __restrict__ t_final) {
    if (*a.status != SQ_OK) return;
    const int lane = threadIdx.x & 31;
    const int s = lane & (GS - 1), gbase = lane & ~(GS - 1);
    const float4* lp4 = reinterpret_cast<const float4*>(a.lpad);

    int rn = 0;
    if (s == 0) rn = atomicAdd(a.ray_ctr, 1);
    long long r = __shfl_sync(0xffffffffu, rn, gbase);
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f};
    if (r < a.R) ray_of(a, r, o, d);
    float T = 1.f, Dp = 0.f;
    int j0 = 0, used_total = 0;
    bool seen_inside = false;
    float acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = 0.f;

    while (__any_sync(0xffffffffu, r < a.R)) {
        const bool live = r < a.R;
        const int j = j0 + s;
        const bool valid = live && j < a.L;
        float x[3] = {0.f, 0.f, 0.f};
        int vox = -1;
        float tj = 0.f;
        if (valid) {
            tj = __ldg(a.t + j);
            vox = sample_voxel(a.g, o, d, tj, x);
        }
        int n = 0, f = 0;
        if (vox >= 0) {
            n = __ldg(a.v_n + vox);
            f = __ldg(a.v_f + vox);
        }
        float asum = 0.f;
        float sacc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) sacc[c] = 0.f;
        const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)n);
        for (int e = 0; e < nmax; ++e) {
            if (e < n) {
                const int k = __ldg(a.v_sq + f + e);
                const Prim p = load_prim(a.rec, k);
                const float po = occupancy(p, x);
                asum = fmaf(po, p.sigma, asum);
                const float4* cr = lp4 + (size_t)k * (CP / 4);
#pragma unroll
                for (int q = 0; q < CP / 4; ++q) {
                    const float4 cv = __ldg(cr + q);
                    sacc[4 * q + 0] = fmaf(po, cv.x, sacc[4 * q + 0]);
                    sacc[4 * q + 1] = fmaf(po, cv.y, sacc[4 * q + 1]);
                    sacc[4 * q + 2] = fmaf(po, cv.z, sacc[4 * q + 2]);
                    sacc[4 * q + 3] = fmaf(po, cv.w, sacc[4 * q + 3]);
                }
            }
        }
        const float alpha = valid ? fminf(asum, a.alpha_max) : 0.f;
        float Tb;
        int used;
        bool stop;
        const float w = group_composite(alpha, s, gbase, a.kappa, T, Tb, valid, used, stop);
        if (valid) {
            if (s < used && a.save_T) a.save_T[r * a.L + j] = Tb;
            Dp = fmaf(w, tj, Dp);
#pragma unroll
            for (int c = 0; c < CP; ++c) acc[c] = fmaf(w, sacc[c], acc[c]);
        }
        // the group's samples: inside the grid anywhere?  t is non-decreasing, so a
        // chunk fully outside after an inside one means the ray has left for good
        const unsigned ins = (__ballot_sync(0xffffffffu, vox >= 0) >> gbase) & ((1u << GS) - 1u);
        const bool left = seen_inside && ins == 0u;
        seen_inside = seen_inside || ins != 0u;
        if (live) used_total = min(j0 + used, a.L);
        j0 += GS;
        // a ray ends at L, on early termination, once T is exactly 0 (every later
        // weight is 0), or when it has left the grid
        const bool fin = live && (j0 >= a.L || stop || T == 0.f || left);
        if (__any_sync(0xffffffffu, fin)) {
            float Dsum = Dp;
#pragma unroll
            for (int o2 = GS / 2; o2 > 0; o2 >>= 1) Dsum += __shfl_xor_sync(0xffffffffu, Dsum, o2, GS);
#pragma unroll
            for (int c = 0; c < CP; ++c) {
                float v = acc[c];
#pragma unroll
                for (int o2 = GS / 2; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2, GS);
                if (fin && (c % GS) == s && c < a.C) sem[r * a.C + c] = v;
            }
            if (fin && s == 0) {
                depth[r] = Dsum;
                if (t_final) t_final[r] = T;
                if (a.save_n) a.save_n[r] = used_total;
            }
            int nr = 0;
            if (fin && s == 0) nr = atomicAdd(a.ray_ctr, 1);
            nr = __shfl_sync(0xffffffffu, nr, gbase);
            if (fin) {
                r = nr;
                if (r < a.R) ray_of(a, r, o, d);
                T = 1.f;
                Dp = 0.f;
                j0 = 0;
                used_total = 0;
                seen_inside = false;
#pragma unroll
                for (int c = 0; c < CP; ++c) acc[c] = 0.f;
            }
        }
    }
}

// ------------------------------------------------------------------ backward
struct BwdPrim {
    Prim f;
    float is[3];  // 1 / s
    float ie1, ie2;
};

__device__ __forceinline__ BwdPrim load_bwd(const float4* __restrict__ rec, const float4* __restrict__ aux, int k) {
    BwdPrim b;
    b.f = load_prim(rec, k);
    const float4* a = aux + (size_t)k * AUX4;
    const float4 a1 = __ldg(a + 1), a2 = __ldg(a + 2);
    b.is[0] = a1.y; b.is[1] = a1.z; b.is[2] = a1.w;
    b.ie1 = a2.z; b.ie2 = a2.w;
    return b;
}

// Per-pair partial derivatives of f, in the form that is summed per (ray,
// primitive) and turned into parameter gradients once at the flush:
//   r[0..2]  gx = df/dx (world), so df/dm = -gx
//   r[3..5]  tau = gx x (x - m), the torque of a world-frame rotation of the primitive
//   r[6..8]  u_j df/du_j, so df/ds_j = -(u_j df/du_j) / s_j
//   r[9..10] df/deps1, df/deps2
// with u_j = (R^T (x - m))_j / s_j, a = |u_0|, b = |u_1|, c = |u_2|,
// f = A^eb + c^ec, A = a^ea + b^ea (ea = 2/eps2, eb = eps2/eps1, ec = 2/eps1).
// Returns p_o = exp(-f).
__device__ __forceinline__ float occupancy_partials(const BwdPrim& P, const float x[3], float r[11]) {
    const Prim& p = P.f;
    const float d[3] = {x[0] - p.m[0], x[1] - p.m[1], x[2] - p.m[2]};
    float u[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) u[j] = fmaf(p.M[j][0], d[0], fmaf(p.M[j][1], d[1], p.M[j][2] * d[2]));
    const float la = lg2(fabsf(u[0])), lb = lg2(fabsf(u[1])), lc = lg2(fabsf(u[2]));
    const float pa = ex2(p.ea * la), pb = ex2(p.ea * lb), pc = ex2(p.ec * lc);
    const float A = pa + pb;
    const float lA = lg2(A);
    const float PA = ex2(p.eb * lA);
    const float po = ex2(-(PA + pc) * LOG2E);
    const float rA = A > 0.f ? rcp(A) : 0.f;
    const float t0 = p.ec * PA * rA;
    r[6] = t0 * pa;
    r[7] = t0 * pb;
    r[8] = p.ec * pc;
    float dfu[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dfu[j] = u[j] != 0.f ? r[6 + j] * rcp(u[j]) : 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = dfu[0] * p.M[0][i] + dfu[1] * p.M[1][i] + dfu[2] * p.M[2][i];
    r[3] = r[1] * d[2] - r[2] * d[1];
    r[4] = r[2] * d[0] - r[0] * d[2];
    r[5] = r[0] * d[1] - r[1] * d[0];
    const float e1term = (PA > 0.f ? p.eb * PA * lA : 0.f) + (pc > 0.f ? p.ec * pc * lc : 0.f);
    r[9] = -LN2 * P.ie1 * e1term;
    const float pl = (pa > 0.f ? pa * la : 0.f) + (pb > 0.f ? pb * lb : 0.f);
    r[10] = PA > 0.f ? PA * LN2 * (lA * P.ie1 - p.ec * P.ie2 * pl * rA) : 0.f;
    return po;
}

struct BwdArgs {
    RenderArgs r;
    const float* grad_depth;
    const float* grad_sem;
    const int4* boxes;  // [N] voxel boxes of the index, 16-bit packed (lo | hi << 16 per axis)
    float* gacc;        // [N, GF] gradient accumulator, zeroed before the launch
};

template <int CP>
__device__ __forceinline__ float logit_dot(const float* __restrict__ lpad, int k, const float* __restrict__ gS, int C) {
    const float4* cr = reinterpret_cast<const float4*>(lpad) + (size_t)k * (CP / 4);
    float cd = 0.f;
#pragma unroll
    for (int q = 0; q < CP / 4; ++q) {
        const float4 c4 = __ldg(cr + q);
        const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * q + i < C) cd = fmaf(__ldg(gS + 4 * q + i), cc[i], cd);
    }
    return cd;
}

// <gS, c_k> with gS staged in shared memory (zero-padded to CP).
template <int CP>
__device__ __forceinline__ float logit_dot_sh(const float* __restrict__ lpad, int k, const float* gS) {
    const float4* cr = reinterpret_cast<const float4*>(lpad) + (size_t)k * (CP / 4);
    float cd = 0.f;
#pragma unroll
    for (int q = 0; q < CP / 4; ++q) {
        const float4 c4 = __ldg(cr + q);
        cd = fmaf(gS[4 * q + 0], c4.x, cd);
        cd = fmaf(gS[4 * q + 1], c4.y, cd);
        cd = fmaf(gS[4 * q + 2], c4.z, cd);
        cd = fmaf(gS[4 * q + 3], c4.w, cd);
    }
    return cd;
}

// Writes the warp's pending flushes into the accumulator of raw partial sums:
// per entry, lane f adds field f (and f + 32).  Fields 0-11 are the summed
// partials (gx 3, tau 3, u df/du 3, eps 2, sigma 1), 12.. the logit gradients
// W gS_c; gsl[b] = gS[32 b + lane - 12] of the current ray.
__device__ __forceinline__ void drain_queue(float* __restrict__ gacc, const float* __restrict__ q, int qn, int lane,
                                            const float gsl[2], int C) {
    for (int e = 0; e < qn; ++e) {
        const float* ent = q + e * QW;
        const int k = __float_as_int(ent[0]);
        float* row = gacc + (size_t)k * GF;
        float v = 0.f;
        if (lane < NRAW) v = ent[1 + lane];
        else if (lane < NRAW + C) v = ent[1 + NRAW] * gsl[0];
        if (v != 0.f) red_add(row + lane, v);
        if (lane + 32 < NRAW + C) {
            const float v2 = ent[1 + NRAW] * gsl[1];
            if (v2 != 0.f) red_add(row + 32 + lane, v2);
        }
    }
}

struct WarpBwd {
    float queue[QCAP * QW];
    float gs[32];  // dL/dS of the current ray
};

// Packed inclusive box test; an empty box is stored as lo = 1, hi = 0.
__device__ __forceinline__ bool box_has(const int4 b, int ix, int iy, int iz) {
    return ix >= (b.x & 0xffff) && ix <= (b.x >> 16) && iy >= (b.y & 0xffff) && iy <= (b.y >> 16) &&
           iz >= (b.z & 0xffff) && iz <= (b.z >> 16);
}

__device__ __forceinline__ int4 shfl_box(int4 b, int src) {
    return make_int4(__shfl_sync(0xffffffffu, b.x, src), __shfl_sync(0xffffffffu, b.y, src),
                     __shfl_sync(0xffffffffu, b.z, src), 0);
}

__global__ void k_pack_boxes(const int* __restrict__ ranges, int n, int4* __restrict__ boxes) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int* r = ranges + 6 * k;
    int v[3];
    const bool empty = r[1] < r[0] || r[3] < r[2] || r[5] < r[4];
    for (int a = 0; a < 3; ++a) v[a] = empty ? 1 : (r[2 * a] | (r[2 * a + 1] << 16));
    boxes[k] = make_int4(v[0], v[1], v[2], 0);
}

// Per-lane state of one owner slot.
struct Slot {
    int key;      // primitive id, -1 when free
    int4 box;     // its voxel box (packed)
    float cd;     // <gS, c_key> of the current ray
    float acc[13];
};

// Pending flush queue of a warp (per-(ray, primitive) partial sums).
struct FlushQ {
    float* q;
    int n;
};

__device__ __forceinline__ void queue_make_room(FlushQ& Q, unsigned dm, float* gacc, int lane, const float gsl[2],
                                                int C, const float4* aux) {
    if (Q.n + __popc(dm) > QCAP) {
        __syncwarp();
        drain_queue(gacc, Q.q, Q.n, lane, gsl, C);
        __syncwarp();
        Q.n = 0;
    }
}

__device__ __forceinline__ void queue_push(FlushQ& Q, bool mine, unsigned dm, unsigned lt, int key, const float v[13]) {
    if (mine) {
        float* ent = Q.q + (Q.n + __popc(dm & lt)) * QW;
        ent[0] = __int_as_float(key);
#pragma unroll
        for (int i = 0; i < 13; ++i) ent[1 + i] = v[i];
    }
    Q.n += __popc(dm);
}

// Owner of slot S leaves when `del`; its sums are queued and the slot freed.
__device__ __forceinline__ void slot_leave(Slot& S, bool del, FlushQ& Q, float* gacc, int lane, unsigned lt,
                                           const float gsl[2], int C, const float4* aux) {
    const unsigned dm = __ballot_sync(0xffffffffu, del);
    if (!dm) return;
    queue_make_room(Q, dm, gacc, lane, gsl, C, aux);
    queue_push(Q, del, dm, lt, S.key, S.acc);
    if (del) S.key = -1;
}

__device__ __forceinline__ void slot_copy_from(Slot& dst, const Slot& src_lane_slot, int src, bool take) {
    const int k = __shfl_sync(0xffffffffu, src_lane_slot.key, src);
    const float c = __shfl_sync(0xffffffffu, src_lane_slot.cd, src);
    int4 b;
    float v[13];
    b.x = __shfl_sync(0xffffffffu, src_lane_slot.box.x, src);
    b.y = __shfl_sync(0xffffffffu, src_lane_slot.box.y, src);
    b.z = __shfl_sync(0xffffffffu, src_lane_slot.box.z, src);
    b.w = 0;
#pragma unroll
    for (int i = 0; i < 13; ++i) v[i] = __shfl_sync(0xffffffffu, src_lane_slot.acc[i], src);
    if (take) {
        dst.key = k;
        dst.cd = c;
        dst.box = b;
#pragma unroll
        for (int i = 0; i < 13; ++i) dst.acc[i] = v[i];
    }
}

template <int CP>
__device__ __forceinline__ void slot_enter(Slot& S, int k, int4 box, const float* __restrict__ lpad,
                                           const float* __restrict__ gS, int C) {
    S.key = k;
    S.box = box;
#pragma unroll
    for (int i = 0; i < 13; ++i) S.acc[i] = 0.f;
    S.cd = logit_dot_sh<CP>(lpad, k, gS);
}

// Evaluates the slot's pair at x: p_o and partials (kept for the accumulation
// once G_j is known) and the slot's share of alpha_j and <gS, s_j>.
__device__ __forceinline__ void slot_eval(const Slot& S, const RenderArgs& a, const float x[3], float& po, float pr[11],
                                          float& sig, float& pa, float& pv) {
    po = 0.f;
    sig = 0.f;
    if (S.key >= 0) {
        const BwdPrim P = load_bwd(a.rec, a.aux, S.key);
        po = occupancy_partials(P, x, pr);
        sig = P.f.sigma;
        pa = fmaf(po, sig, pa);
        pv = fmaf(po, S.cd, pv);
    }
}

__device__ __forceinline__ void slot_accumulate(Slot& S, float po, const float pr[11], float sig, float G, float w) {
    if (S.key >= 0 && po != 0.f) {
        const float gf = -po * fmaf(G, sig, w * S.cd);
#pragma unroll
        for (int i = 0; i < 11; ++i) S.acc[i] = fmaf(gf, pr[i], S.acc[i]);
        S.acc[11] = fmaf(G, po, S.acc[11]);
        S.acc[12] = fmaf(w, po, S.acc[12]);
    }
}

// One warp per ray, samples back to front (Sec. 3.3.3).  With T_j saved by the
// forward, U_j is carried from the back, so one sweep gives alpha_j, v_j, G_j and
// every pair's gradient.  Owner bookkeeping uses the primitives' voxel boxes: an
// owner leaves when the sample's voxel is outside its box, and a list entry is new
// when the previous sample's voxel is outside its box.
template <int CP>
__global__ void __launch_bounds__(BWD_WARPS * 32, 2) k_backward(BwdArgs A) {
    __shared__ WarpBwd smem[BWD_WARPS];
    const RenderArgs& a = A.r;
    if (*a.status != SQ_OK) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float* gSs = smem[wid].gs;

    for (;;) {
        int rr = 0;
        if (lane == 0) rr = atomicAdd(a.ray_ctr, 1);
        const long long r = __shfl_sync(0xffffffffu, rr, 0);
        if (r >= a.R) break;
        const int Le = __ldg(a.save_n + r);
        __syncwarp();
        gSs[lane] = lane < a.C ? __ldg(A.grad_sem + r * a.C + lane) : 0.f;
        __syncwarp();
        float o[3], d[3];
        ray_of(a, r, o, d);
        const float gD = __ldg(A.grad_depth + r);
        const float* gS = A.grad_sem + r * a.C;
        float gsl[2];
        gsl[0] = (lane >= NRAW && lane < NRAW + a.C) ? __ldg(gS + (lane - NRAW)) : 0.f;
        gsl[1] = (lane + 32 < NRAW + a.C) ? __ldg(gS + (lane + 32 - NRAW)) : 0.f;

        Slot S0, S1;
        S0.key = -1;
        S1.key = -1;
        FlushQ Q{smem[wid].queue, 0};
        float U = 0.f;
        int pvx = -1, piy = 0, piz = 0, pvox = -1;  // voxel of the previously processed sample (-1: none)

        for (int j = Le - 1; j >= -1; --j) {
            // j == -1: an empty list releases every owner
            int n = 0, f = 0, vox = -1, ix = -1, iy = 0, iz = 0;
            float x[3] = {0.f, 0.f, 0.f};
            float tj = 0.f;
            if (j >= 0) {
                tj = __ldg(a.t + j);
                int vi[3];
                vox = sample_voxel(a.g, o, d, tj, x, vi);
                if (vox >= 0) {
                    n = __ldg(a.v_n + vox);
                    f = __ldg(a.v_f + vox);
                    ix = vi[0];
                    iy = vi[1];
                    iz = vi[2];
                }
            }
            const bool heavy = n > OWN;
            if (vox != pvox || heavy) {
                // owners whose box misses this voxel leave (all of them on an empty or heavy list)
                const bool gone = n == 0 || heavy;
                slot_leave(S0, S0.key >= 0 && (gone || !box_has(S0.box, ix, iy, iz)), Q, A.gacc, lane, lt, gsl, a.C,
                           a.aux);
                slot_leave(S1, S1.key >= 0 && (gone || !box_has(S1.box, ix, iy, iz)), Q, A.gacc, lane, lt, gsl, a.C,
                           a.aux);
                if (!gone) {
                    // slot-1 owners move to free slot-0 lanes
                    const unsigned o1 = __ballot_sync(0xffffffffu, S1.key >= 0);
                    if (SQR_MIGRATE && o1) {
                        const unsigned f0 = __ballot_sync(0xffffffffu, S0.key < 0);
                        const int mv = __popc(o1);
                        if (mv <= __popc(f0)) {
                            const int rk = __popc(f0 & lt);
                            const bool take = S0.key < 0 && rk < mv;
                            const int src = take ? __fns(o1, 0, rk + 1) : lane;
                            const bool given = S1.key >= 0 && __popc(o1 & lt) < mv;
                            slot_copy_from(S0, S1, src, take);
                            if (given) S1.key = -1;
                        }
                    }
                    // list entries whose box misses the previous voxel are new owners
                    int kn0 = -1, kn1 = -1;
                    int4 bx0 = make_int4(1, 1, 1, 0), bx1 = make_int4(1, 1, 1, 0);
                    bool new0 = false, new1 = false;
                    if (lane < n) {
                        kn0 = __ldg(a.v_sq + f + lane);
                        bx0 = __ldg(A.boxes + kn0);
                        new0 = pvox < 0 || !box_has(bx0, pvx, piy, piz);
                    }
                    if (lane + 32 < n) {
                        kn1 = __ldg(a.v_sq + f + lane + 32);
                        bx1 = __ldg(A.boxes + kn1);
                        new1 = pvox < 0 || !box_has(bx1, pvx, piy, piz);
                    }
                    const unsigned nm0 = __ballot_sync(0xffffffffu, new0), nm1 = __ballot_sync(0xffffffffu, new1);
                    const int c0 = __popc(nm0), nnew = c0 + __popc(nm1);
                    if (nnew) {
                        const unsigned fr0 = __ballot_sync(0xffffffffu, S0.key < 0);
                        const unsigned fr1 = __ballot_sync(0xffffffffu, S1.key < 0);
                        {
                            const int rk = __popc(fr0 & lt);
                            const bool want = S0.key < 0 && rk < nnew;
                            int src = lane;
                            bool hi = false;
                            if (want) {
                                if (rk < c0) src = __fns(nm0, 0, rk + 1);
                                else { src = __fns(nm1, 0, rk - c0 + 1); hi = true; }
                            }
                            const int va = __shfl_sync(0xffffffffu, kn0, src);
                            const int vb = __shfl_sync(0xffffffffu, kn1, src);
                            const int4 ba = shfl_box(bx0, src), bb1 = shfl_box(bx1, src);
                            const int4 bb = hi ? bb1 : ba;
                            if (want) slot_enter<CP>(S0, hi ? vb : va, bb, a.lpad, gSs, a.C);
                        }
                        if (nnew > __popc(fr0)) {
                            const int rk = __popc(fr0) + __popc(fr1 & lt);
                            const bool want = S1.key < 0 && rk < nnew;
                            int src = lane;
                            bool hi = false;
                            if (want) {
                                if (rk < c0) src = __fns(nm0, 0, rk + 1);
                                else { src = __fns(nm1, 0, rk - c0 + 1); hi = true; }
                            }
                            const int va = __shfl_sync(0xffffffffu, kn0, src);
                            const int vb = __shfl_sync(0xffffffffu, kn1, src);
                            const int4 ba = shfl_box(bx0, src), bb1 = shfl_box(bx1, src);
                            const int4 bb = hi ? bb1 : ba;
                            if (want) slot_enter<CP>(S1, hi ? vb : va, bb, a.lpad, gSs, a.C);
                        }
                    }
                }
                pvox = gone ? -1 : vox;
                pvx = ix; piy = iy; piz = iz;
            }
            if (j < 0) break;
            if (n == 0) continue;  // no primitive here: alpha_j = 0 leaves U unchanged
            float po0, po1 = 0.f, pr0[11], pr1[11], sg0, sg1 = 0.f;
            float pa = 0.f, pv = 0.f;
            slot_eval(S0, a, x, po0, pr0, sg0, pa, pv);
            const bool any1 = __any_sync(0xffffffffu, S1.key >= 0);
            if (any1) slot_eval(S1, a, x, po1, pr1, sg1, pa, pv);
            if (heavy) {
                for (int e = lane; e < n; e += 32) {
                    const int k = __ldg(a.v_sq + f + e);
                    const Prim p = load_prim(a.rec, k);
                    const float pe = occupancy(p, x);
                    pa = fmaf(pe, p.sigma, pa);
                    pv = fmaf(pe, logit_dot<CP>(a.lpad, k, gS, a.C), pv);
                }
            }
            const float raw = warp_sum(pa);
            const float vs = warp_sum(pv);
            const float alpha = fminf(raw, a.alpha_max);
            const float Tj = __ldg(a.save_T + r * a.L + j);
            const float vj = fmaf(gD, tj, vs);
            const float G = raw > a.alpha_max ? 0.f : Tj * (vj - U);  // dL/dalpha_j
            const float w = Tj * alpha;
            slot_accumulate(S0, po0, pr0, sg0, G, w);
            if (any1) slot_accumulate(S1, po1, pr1, sg1, G, w);
            if (heavy) {
                // every pair of a heavy list is queued on its own
                for (int e0 = 0; e0 < n; e0 += 32) {
                    const int e = e0 + lane;
                    float v[13];
                    int k = -1;
                    bool mine = false;
                    if (e < n) {
                        k = __ldg(a.v_sq + f + e);
                        const BwdPrim P = load_bwd(a.rec, a.aux, k);
                        float pp[11];
                        const float pe = occupancy_partials(P, x, pp);
                        const float gf = -pe * fmaf(G, P.f.sigma, w * logit_dot<CP>(a.lpad, k, gS, a.C));
#pragma unroll
                        for (int i = 0; i < 11; ++i) v[i] = gf * pp[i];
                        v[11] = G * pe;
                        v[12] = w * pe;
                        mine = pe != 0.f;
                    }
                    const unsigned dm = __ballot_sync(0xffffffffu, mine);
                    if (dm) {
                        queue_make_room(Q, dm, A.gacc, lane, gsl, a.C, a.aux);
                        queue_push(Q, mine, dm, lt, k, v);
                    }
                }
            }
            U = fmaf(alpha, vj, (1.f - alpha) * U);
        }
        __syncwarp();
        drain_queue(A.gacc, Q.q, Q.n, lane, gsl, a.C);
        __syncwarp();
    }
}

// Converts each primitive's summed partials into the six gradient outputs:
//   dL/dm = -sum gx;  dL/dq = (0, 2 tau) (x) qn / |q| (the torque of a world-frame
//   rotation mapped onto the tangent of the unit quaternion, then through q/|q|);
//   dL/ds_j = -sum(u_j df/du_j) / s_j;  dL/deps, dL/dsigma as summed;
//   dL/dc as accumulated.  One thread per primitive.
__global__ void k_grad_out(const float* __restrict__ gacc, const float4* __restrict__ aux, int n, int C,
                           float* __restrict__ gm, float* __restrict__ gq, float* __restrict__ gs,
                           float* __restrict__ ge, float* __restrict__ go, float* __restrict__ gl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float* e = gacc + (size_t)k * GF;
    const float4 a0 = aux[(size_t)k * AUX4], a1 = aux[(size_t)k * AUX4 + 1];
    const float w = a0.x, v[3] = {a0.y, a0.z, a0.w}, inq = a1.x, is[3] = {a1.y, a1.z, a1.w};
    for (int i = 0; i < 3; ++i) gm[3 * k + i] = -e[i];
    const float t[3] = {e[3], e[4], e[5]};
    gq[4 * k + 0] = -2.f * (t[0] * v[0] + t[1] * v[1] + t[2] * v[2]) * inq;
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        gq[4 * k + 1 + i] = 2.f * (w * t[i] + t[i1] * v[i2] - t[i2] * v[i1]) * inq;
    }
    for (int i = 0; i < 3; ++i) gs[3 * k + i] = -e[6 + i] * is[i];
    ge[2 * k + 0] = e[9];
    ge[2 * k + 1] = e[10];
    go[k] = e[11];
    for (int c = 0; c < C; ++c) gl[(size_t)k * C + c] = e[NRAW + c];
}

// ------------------------------------------------------------------ pair counter
__global__ void __launch_bounds__(256) k_count_pairs(RenderArgs a, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long sq[8], ss[8];
    unsigned long long q = 0, s = 0;
    const long long total = a.R * a.L;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / a.L;
        const int j = (int)(e - r * a.L);
        float o[3], d[3], x[3];
        ray_of(a, r, o, d);
        int vox = sample_voxel(a.g, o, d, __ldg(a.t + j), x);
        if (vox >= 0) {
            q += (unsigned long long)__ldg(a.v_n + vox);
            s += 1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        q += __shfl_xor_sync(0xffffffffu, q, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sq[threadIdx.x >> 5] = q;
        ss[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tq = 0, ts = 0;
        for (int w = 0; w < 8; ++w) { tq += sq[w]; ts += ss[w]; }
        atomicAdd(out, tq);
        atomicAdd(out + 1, ts);
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
    return sms;
}

sq_status_t count_pairs_impl(const sq_index_t* idx, const sq_grid_t* grid, const sq_rays_t* rays, long long* out,
                             cudaStream_t st) {
    RenderArgs a{};
    a.v_n = idx->v_n;
    a.g = make_grid(grid);
    a.K = rays->K;
    a.c2w = rays->cam2world;
    a.t = rays->t;
    a.n_cam = rays->n_cam;
    a.H = rays->H;
    a.W = rays->W;
    a.L = rays->L;
    a.R = (long long)rays->n_cam * rays->H * rays->W;
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(long long), st);
    if (e != cudaSuccess) return cuda_status(e, "memset count");
    if (a.R == 0) return SQ_OK;
    long long want = (a.R * a.L + 255) / 256;
    int blocks = (int)(want < 152LL * 16 ? want : 152LL * 16);
    k_count_pairs<<<blocks, 256, 0, st>>>(a, reinterpret_cast<unsigned long long*>(out));
    SQ_CHECK_LAUNCH("k_count_pairs");
    return SQ_OK;
}

sq_status_t launch_pack(const sq_prims_t* prims, float4* rec, float4* aux, float* lpad, int cp, cudaStream_t st) {
    if (prims->n == 0) return SQ_OK;
    k_pack<<<(prims->n + 127) / 128, 128, 0, st>>>(*prims, rec, aux, lpad, cp);
    SQ_CHECK_LAUNCH("k_pack");
    return SQ_OK;
}

// Render workspace: packed records, backward extras, padded logits, gradient
// accumulator [N, 32] and the work counter.
struct RenderWs {
    size_t rec_off, aux_off, lpad_off, gacc_off, box_off, ctr_off, total;
};

static RenderWs render_ws(const sq_prims_t* p) {
    RenderWs w;
    const size_t n = (size_t)(p->n > 0 ? p->n : 0);
    const int cp = cpad(p->n_classes);
    w.rec_off = 0;
    w.aux_off = align_up(n * REC4 * sizeof(float4), 256);
    w.lpad_off = align_up(w.aux_off + n * AUX4 * sizeof(float4), 256);
    w.gacc_off = align_up(w.lpad_off + n * cp * sizeof(float), 256);
    w.box_off = align_up(w.gacc_off + n * GF * sizeof(float), 256);
    w.ctr_off = align_up(w.box_off + n * sizeof(int4), 256);
    w.total = w.ctr_off + 256;
    return w;
}

size_t render_workspace_size(const sq_prims_t* p) { return render_ws(p).total; }

size_t render_logits_offset(const sq_prims_t* p) { return render_ws(p).lpad_off; }

static sq_status_t setup_render(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                                const sq_rays_t* rays, void* ws, size_t ws_bytes, cudaStream_t st, bool need_aux,
                                RenderArgs& a, float** gacc, const char* who) {
    RenderWs w = render_ws(prims);
    if (ws == nullptr || ws_bytes < w.total) {
        set_last_error("%s: workspace of %zu bytes given, %zu needed", who, ws_bytes, w.total);
        return SQ_ERR_INVALID_ARG;
    }
    const long long R = (long long)rays->n_cam * rays->H * rays->W;
    if (R >= 2147483647LL - 64) {
        set_last_error("%s: %lld rays, at most 2^31 - 64 supported per call", who, R);
        return SQ_ERR_INVALID_ARG;
    }
    char* base = (char*)ws;
    float4* rec = (float4*)(base + w.rec_off);
    float4* aux = need_aux ? (float4*)(base + w.aux_off) : nullptr;
    float* lpad = (float*)(base + w.lpad_off);
    const int cp = cpad(prims->n_classes);
    sq_status_t s = launch_pack(prims, rec, aux, lpad, cp, st);
    if (s != SQ_OK) return s;
    cudaError_t e = cudaMemsetAsync(base + w.ctr_off, 0, 256, st);
    if (e != cudaSuccess) return cuda_status(e, "memset counter");
    a.rec = rec;
    a.aux = (float4*)(base + w.aux_off);
    a.lpad = lpad;
    a.v_n = idx->v_n;
    a.v_f = idx->v_f;
    a.v_sq = idx->v_sq;
    a.status = idx->status;
    a.g = make_grid(grid);
    a.K = rays->K;
    a.c2w = rays->cam2world;
    a.t = rays->t;
    a.n_cam = rays->n_cam;
    a.H = rays->H;
    a.W = rays->W;
    a.L = rays->L;
    a.C = prims->n_classes;
    a.R = R;
    a.kappa = rays->kappa;
    a.alpha_max = rays->alpha_max;
    a.ray_ctr = (int*)(base + w.ctr_off);
    a.save_T = nullptr;
    a.save_n = nullptr;
    if (gacc) *gacc = (float*)(base + w.gacc_off);
    a.boxes = (int4*)(base + w.box_off);
    return SQ_OK;
}

// Saved forward state: T [R, L] (transmittance before each sample) then n [R].
size_t saved_size(const sq_rays_t* r) {
    const size_t R = (size_t)r->n_cam * r->H * r->W;
    return align_up(R * r->L * sizeof(float), 256) + align_up(R * sizeof(int), 256);
}

static void saved_ptrs(const sq_rays_t* r, void* saved, float** T, int** n) {
    const size_t R = (size_t)r->n_cam * r->H * r->W;
    *T = (float*)saved;
    *n = (int*)((char*)saved + align_up(R * r->L * sizeof(float), 256));
}

template <int CP>
static sq_status_t launch_persistent(const void* fn, int threads, size_t smem, long long work, int per_block,
                                     void** args, cudaStream_t st, const char* who) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return cuda_status(e, who);
    long long need = (work + per_block - 1) / per_block;
    long long blocks = (long long)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(threads), args, smem, st);
    if (e != cudaSuccess) return cuda_status(e, who);
    return SQ_OK;
}

template <int CP>
static sq_status_t launch_fwd_cp(RenderArgs a, float* depth, float* sem, float* t_final, cudaStream_t st) {
    void* args[] = {&a, &depth, &sem, &t_final};
    return launch_persistent<CP>((const void*)k_forward<CP>, FWD_WARPS * 32, 0, a.R, FWD_WARPS * 4, args, st,
                                 "k_forward");
}

#define SQ_DISPATCH_CP(cp, CALL)                          \
    switch (cp) {                                         \
        case 4: { constexpr int CPV = 4; return CALL; }   \
        case 8: { constexpr int CPV = 8; return CALL; }   \
        case 12: { constexpr int CPV = 12; return CALL; } \
        case 16: { constexpr int CPV = 16; return CALL; } \
        case 20: { constexpr int CPV = 20; return CALL; } \
        case 24: { constexpr int CPV = 24; return CALL; } \
        case 28: { constexpr int CPV = 28; return CALL; } \
        case 32: { constexpr int CPV = 32; return CALL; } \
        default: return SQ_ERR_INVALID_ARG;               \
    }

sq_status_t render_fwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* saved,
                            size_t saved_bytes, void* ws, size_t ws_bytes, cudaStream_t st) {
    RenderArgs a;
    if (saved && saved_bytes < saved_size(rays)) {
        set_last_error("sq_render_fwd: saved state of %zu bytes given, %zu needed", saved_bytes, saved_size(rays));
        return SQ_ERR_INVALID_ARG;
    }
    sq_status_t s = setup_render(prims, idx, grid, rays, ws, ws_bytes, st, false, a, nullptr, "sq_render_fwd");
    if (s != SQ_OK) return s;
    if (saved) saved_ptrs(rays, saved, &a.save_T, &a.save_n);
    if (a.R == 0) return SQ_OK;
    const int cp = cpad(prims->n_classes);
    SQ_DISPATCH_CP(cp, (launch_fwd_cp<CPV>(a, depth, sem, t_final, st)));
}

template <int CP>
static sq_status_t launch_bwd_cp(BwdArgs A, cudaStream_t st) {
    void* args[] = {&A};
    return launch_persistent<CP>((const void*)k_backward<CP>, BWD_WARPS * 32, 0, A.r.R, BWD_WARPS, args, st,
                                 "k_backward");
}

sq_status_t render_bwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, const void* saved, size_t saved_bytes, const float* grad_depth,
                            const float* grad_sem, float* g_means, float* g_quats, float* g_scales, float* g_eps,
                            float* g_opacity, float* g_logits, void* ws, size_t ws_bytes, cudaStream_t st) {
    BwdArgs A;
    if (!saved || saved_bytes < saved_size(rays)) {
        set_last_error("sq_render_bwd: saved state of %zu bytes given, %zu needed", saved_bytes, saved_size(rays));
        return SQ_ERR_INVALID_ARG;
    }
    float* gacc = nullptr;
    sq_status_t s = setup_render(prims, idx, grid, rays, ws, ws_bytes, st, true, A.r, &gacc, "sq_render_bwd");
    if (s != SQ_OK) return s;
    saved_ptrs(rays, const_cast<void*>(saved), &A.r.save_T, &A.r.save_n);
    const int n = prims->n;
    const int C = prims->n_classes;
    if (n == 0) return SQ_OK;
    cudaError_t e = cudaMemsetAsync(gacc, 0, (size_t)n * GF * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "memset gradient accumulator");
    A.grad_depth = grad_depth;
    A.grad_sem = grad_sem;
    A.boxes = A.r.boxes;
    A.gacc = gacc;
    if (grid->nx > 65535 || grid->ny > 65535 || grid->nz > 65535) {
        set_last_error("sq_render_bwd: grid dims above 65535 per axis are not supported");
        return SQ_ERR_INVALID_ARG;
    }
    k_pack_boxes<<<(n + 127) / 128, 128, 0, st>>>(idx->ranges, n, A.r.boxes);
    SQ_CHECK_LAUNCH("k_pack_boxes");
    if (A.r.R > 0) {
        const int cp = cpad(C);
        sq_status_t ls;
        switch (cp) {
            case 4: ls = launch_bwd_cp<4>(A, st); break;
            case 8: ls = launch_bwd_cp<8>(A, st); break;
            case 12: ls = launch_bwd_cp<12>(A, st); break;
            case 16: ls = launch_bwd_cp<16>(A, st); break;
            case 20: ls = launch_bwd_cp<20>(A, st); break;
            case 24: ls = launch_bwd_cp<24>(A, st); break;
            case 28: ls = launch_bwd_cp<28>(A, st); break;
            case 32: ls = launch_bwd_cp<32>(A, st); break;
            default: return SQ_ERR_INVALID_ARG;
        }
        if (ls != SQ_OK) return ls;
    }
    k_grad_out<<<(n + 127) / 128, 128, 0, st>>>(gacc, A.r.aux, n, C, g_means, g_quats, g_scales, g_eps, g_opacity,
                                                g_logits);
    SQ_CHECK_LAUNCH("k_grad_out");
    return SQ_OK;
}

}  // namespace sqr
