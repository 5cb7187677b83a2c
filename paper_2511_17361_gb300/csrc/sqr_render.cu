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

constexpr int GS = 8;         // lanes (samples) per ray in the lane-per-sample layout
constexpr int NG = 32 / GS;   // rays per warp in that layout
constexpr int FWD_WARPS = 8;  // warps per CTA, forward
constexpr int OWN = 64;       // owner slots per warp (two per lane)
constexpr int QCAP = 64;      // pending gradient flushes per warp
constexpr int QW = 16;        // words per pending flush: key, 12 geometry, sigma, W, pad
constexpr int GF = 32;        // floats per primitive in the gradient accumulator
constexpr int NGEO = 13;      // m3 q4 s3 eps2 sigma1

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
    float s[3] = {P.scales[3 * k + 0], P.scales[3 * k + 1], P.scales[3 * k + 2]};
    float e1 = P.eps[2 * k + 0], e2 = P.eps[2 * k + 1];
    float ea = 2.f / e2, eb = e2 / e1, ec = 2.f / e1;
    float M[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) M[j][i] = R[i][j] / s[j];
    float4* r = rec + (size_t)k * REC4;
    r[0] = make_float4(P.means[3 * k + 0], P.means[3 * k + 1], P.means[3 * k + 2], P.opacity[k]);
    r[1] = make_float4(M[0][0], M[0][1], M[0][2], ea);
    r[2] = make_float4(M[1][0], M[1][1], M[1][2], eb);
    r[3] = make_float4(M[2][0], M[2][1], M[2][2], ec);
    if (aux) {
        float4* a = aux + (size_t)k * AUX4;
        a[0] = make_float4(w, x, y, z);
        a[1] = make_float4(inq, s[0], s[1], s[2]);
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
    int* ray_ctr;  // work counter, zeroed before the launch
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
    int j0 = 0;
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
            Dp = fmaf(w, tj, Dp);
#pragma unroll
            for (int c = 0; c < CP; ++c) acc[c] = fmaf(w, sacc[c], acc[c]);
        }
        j0 += GS;
        // a ray ends at L, on early termination, or once T is exactly 0 (every later weight is 0)
        const bool fin = live && (j0 >= a.L || stop || T == 0.f);
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
#pragma unroll
                for (int c = 0; c < CP; ++c) acc[c] = 0.f;
            }
        }
    }
}

// ------------------------------------------------------------------ backward
struct BwdPrim {
    Prim f;
    float qn[4];
    float inv_qn;
    float s[3];
    float e1, e2, ie1, ie2;
};

__device__ __forceinline__ BwdPrim load_bwd(const float4* __restrict__ rec, const float4* __restrict__ aux, int k) {
    BwdPrim b;
    b.f = load_prim(rec, k);
    const float4* a = aux + (size_t)k * AUX4;
    float4 a0 = __ldg(a + 0), a1 = __ldg(a + 1), a2 = __ldg(a + 2);
    b.qn[0] = a0.x; b.qn[1] = a0.y; b.qn[2] = a0.z; b.qn[3] = a0.w;
    b.inv_qn = a1.x; b.s[0] = a1.y; b.s[1] = a1.z; b.s[2] = a1.w;
    b.e1 = a2.x; b.e2 = a2.y; b.ie1 = a2.z; b.ie2 = a2.w;
    return b;
}

// df/d(parameters) at point x.  Outputs p_o and the 12 geometric partials
// g[0..2] = df/dm, g[3..6] = df/dq (raw quaternion), g[7..9] = df/ds, g[10..11] = df/d(eps1, eps2).
__device__ __forceinline__ float occupancy_grad(const BwdPrim& P, const float x[3], float g[12]) {
    const Prim& p = P.f;
    float d[3] = {x[0] - p.m[0], x[1] - p.m[1], x[2] - p.m[2]};
    float u[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) u[j] = fmaf(p.M[j][0], d[0], fmaf(p.M[j][1], d[1], p.M[j][2] * d[2]));
    float la = lg2(fabsf(u[0])), lb = lg2(fabsf(u[1])), lc = lg2(fabsf(u[2]));
    float pa = ex2(p.ea * la), pb = ex2(p.ea * lb), pc = ex2(p.ec * lc);
    float A = pa + pb;
    float lA = lg2(A);
    float PA = ex2(p.eb * lA);
    float f = PA + pc;
    float po = ex2(-f * LOG2E);

    float rA = A > 0.f ? rcp(A) : 0.f;
    float t0 = p.ec * PA * rA;
    float ta = t0 * pa, tb = t0 * pb, tc = p.ec * pc;  // = dfu_j * u_j
    float dfu[3];
    dfu[0] = u[0] != 0.f ? ta * rcp(u[0]) : 0.f;
    dfu[1] = u[1] != 0.f ? tb * rcp(u[1]) : 0.f;
    dfu[2] = u[2] != 0.f ? tc * rcp(u[2]) : 0.f;
    // d f / d x (world) = sum_j dfu_j M_j ; df/dm = -that
    float gd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) gd[i] = dfu[0] * p.M[0][i] + dfu[1] * p.M[1][i] + dfu[2] * p.M[2][i];
    g[0] = -gd[0]; g[1] = -gd[1]; g[2] = -gd[2];
    // scales: u_j = (R^T d)_j / s_j  =>  df/ds_j = -dfu_j u_j / s_j
    g[7] = -ta / P.s[0];
    g[8] = -tb / P.s[1];
    g[9] = -tc / P.s[2];
    // exponents
    float e1term = (PA > 0.f ? p.eb * PA * lA : 0.f) + (pc > 0.f ? p.ec * pc * lc : 0.f);
    g[10] = -LN2 * P.ie1 * e1term;
    float pl = (pa > 0.f ? pa * la : 0.f) + (pb > 0.f ? pb * lb : 0.f);
    g[11] = PA > 0.f ? PA * LN2 * (lA * P.ie1 - p.ec * P.ie2 * pl * rA) : 0.f;
    // rotation: x_S = R^T d, df/dxS_j = dfu_j / s_j, df/dR_ij = d_i df/dxS_j
    float gl[3] = {dfu[0] / P.s[0], dfu[1] / P.s[1], dfu[2] / P.s[2]};
    float gR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) gR[3 * i + j] = d[i] * gl[j];
    const float w = P.qn[0], qx = P.qn[1], qy = P.qn[2], qz = P.qn[3];
    float gq[4];
    gq[0] = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    gq[1] = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - w * gR[5] + qz * gR[6] + w * gR[7] -
                   2.f * qx * gR[8]);
    gq[2] = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] - w * gR[6] + qz * gR[7] -
                   2.f * qy * gR[8]);
    gq[3] = 2.f * (-2.f * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2.f * qz * gR[4] + qy * gR[5] +
                   qx * gR[6] + qy * gR[7]);
    float dot = gq[0] * w + gq[1] * qx + gq[2] * qy + gq[3] * qz;
    g[3] = (gq[0] - w * dot) * P.inv_qn;
    g[4] = (gq[1] - qx * dot) * P.inv_qn;
    g[5] = (gq[2] - qy * dot) * P.inv_qn;
    g[6] = (gq[3] - qz * dot) * P.inv_qn;
    return po;
}


struct BwdArgs {
    RenderArgs r;
    const float* grad_depth;
    const float* grad_sem;
    float* gacc;  // [N, GF] gradient accumulator, zeroed before the launch
};

// Lower-bound membership test in a sorted 64-entry shared array padded with INT_MAX.
__device__ __forceinline__ bool sorted64_has(const int* __restrict__ arr, int key) {
    int pos = 0;
#pragma unroll
    for (int step = 32; step > 0; step >>= 1)
        if (arr[pos + step - 1] < key) pos += step;
    return pos < OWN && arr[pos] == key;
}

template <int CP>
__device__ __forceinline__ float logit_dot(const float* __restrict__ lpad, int k, const float gS[CP]) {
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

// Writes the pending flushes of the warp into the accumulator: one coalesced
// 32-wide atomic add per entry (lane f adds field f).  gsl = gS[lane - 13] of the
// current ray for the logit fields (dL/dc_k = W_k gS).
__device__ __forceinline__ void drain_queue(float* __restrict__ gacc, const float* __restrict__ q, int qn, int lane,
                                            float gsl, int C) {
    for (int e = 0; e < qn; ++e) {
        const float* ent = q + e * QW;
        const int k = __float_as_int(ent[0]);
        float v = 0.f;
        if (lane < NGEO) v = ent[1 + lane];
        else if (lane < NGEO + C) v = ent[1 + NGEO] * gsl;
        if (v != 0.f) red_add(gacc + (size_t)k * GF + lane, v);
    }
}

// Per-warp shared memory of the backward kernel (dynamic; L-dependent part last).
struct WarpBwd {
    int keys[2][OWN];
    float queue[QCAP * QW];
};

template <int CP>
__global__ void __launch_bounds__(256, 2) k_backward(BwdArgs A) {
    extern __shared__ __align__(16) unsigned char dyn[];
    const RenderArgs& a = A.r;
    if (*a.status != SQ_OK) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int s = lane & (GS - 1), gbase = lane & ~(GS - 1), g = lane / GS;
    const int L = a.L;
    WarpBwd& wb = reinterpret_cast<WarpBwd*>(dyn)[wid];
    float* samp = reinterpret_cast<float*>(dyn + (size_t)nw * sizeof(WarpBwd)) + (size_t)wid * NG * 3 * L;
    const unsigned lt = (1u << lane) - 1u;

    for (;;) {
        int r0 = 0;
        if (lane == 0) r0 = atomicAdd(a.ray_ctr, NG);
        r0 = __shfl_sync(0xffffffffu, r0, 0);
        if (r0 >= a.R) break;

        // ------------------------------------------------ phase 1: replay (lane = sample)
        const long long r = (long long)r0 + g;
        const bool live = r < a.R;
        float* sA = samp + (size_t)g * 3 * L;  // +-alpha_j (negative where clamped), then w_j
        float* sV = sA + L;                    // v_j, then G_j = dL/dalpha_j
        float* sT = sA + 2 * L;                // T_j
        float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f};
        float gD = 0.f;
        float gS[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) gS[c] = 0.f;
        if (live) {
            ray_of(a, r, o, d);
            gD = __ldg(A.grad_depth + r);
#pragma unroll
            for (int c = 0; c < CP; ++c)
                if (c < a.C) gS[c] = __ldg(A.grad_sem + r * a.C + c);
        }
        float T = 1.f;
        int j0 = 0, Leff = 0;
        bool run = live;
        while (__any_sync(0xffffffffu, run)) {
            const int j = j0 + s;
            const bool valid = run && j < L;
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
            float asum = 0.f, vsum = 0.f;
            const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)n);
            for (int e = 0; e < nmax; ++e) {
                if (e < n) {
                    const int k = __ldg(a.v_sq + f + e);
                    const Prim p = load_prim(a.rec, k);
                    const float po = occupancy(p, x);
                    asum = fmaf(po, p.sigma, asum);
                    vsum = fmaf(po, logit_dot<CP>(a.lpad, k, gS), vsum);
                }
            }
            const float alpha = valid ? fminf(asum, a.alpha_max) : 0.f;
            float Tb;
            int used;
            bool stop;
            group_composite(alpha, s, gbase, a.kappa, T, Tb, valid, used, stop);
            if (valid && s < used) {
                sA[j] = (asum > a.alpha_max) ? -alpha : alpha;
                sV[j] = fmaf(gD, tj, vsum);
                sT[j] = Tb;
            }
            if (run) {
                Leff = min(j0 + used, L);
                j0 += GS;
                if (j0 >= L || stop || T == 0.f) run = false;
            }
        }
        __syncwarp();
        // ------------------------------------------------ phase 2: back-to-front sweep
        if (live && s == 0) {
            float U = 0.f;
            for (int j = Leff - 1; j >= 0; --j) {
                const float sa = sA[j], vj = sV[j], Tj = sT[j];
                const bool clamped = sa < 0.f;
                const float al = fabsf(sa);
                sV[j] = clamped ? 0.f : Tj * (vj - U);
                U = fmaf(al, vj, (1.f - al) * U);
                sA[j] = Tj * al;
            }
        }
        __syncwarp();
        // ------------------------------------------------ phase 3: gradients (lane = owner)
        for (int gg = 0; gg < NG; ++gg) {
            const long long rr = (long long)r0 + gg;
            if (rr >= a.R) break;
            const int Le = __shfl_sync(0xffffffffu, Leff, gg * GS);
            const float* wA = samp + (size_t)gg * 3 * L;  // w_j
            const float* wG = wA + L;                      // G_j
            float ro[3], rd[3];
            ray_of(a, rr, ro, rd);
            float gSr[CP];
#pragma unroll
            for (int c = 0; c < CP; ++c) gSr[c] = (c < a.C) ? __ldg(A.grad_sem + rr * a.C + c) : 0.f;
            const float gsl = (lane >= NGEO && lane < NGEO + a.C) ? __ldg(A.grad_sem + rr * a.C + (lane - NGEO)) : 0.f;

            int key[2] = {-1, -1};
            float acc[2][14];
            float cdk[2] = {0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int i = 0; i < 14; ++i) acc[q][i] = 0.f;
            int* kold = wb.keys[0];
            int* knew = wb.keys[1];
            kold[lane] = INT_MAX;
            kold[lane + 32] = INT_MAX;
            int qn = 0;
            __syncwarp();

            for (int j = 0; j <= Le; ++j) {
                // j == Le: a final empty list flushes every owner
                float G = 0.f, w = 0.f;
                int n = 0, f = 0;
                float x[3] = {0.f, 0.f, 0.f};
                if (j < Le) {
                    G = wG[j];
                    w = wA[j];
                    if (G == 0.f && w == 0.f) continue;
                    const int vox = sample_voxel(a.g, ro, rd, __ldg(a.t + j), x);
                    if (vox >= 0) {
                        n = __ldg(a.v_n + vox);
                        f = __ldg(a.v_f + vox);
                    }
                }
                const int m = min(n, OWN);
                const int kn0 = lane < m ? __ldg(a.v_sq + f + lane) : INT_MAX;
                const int kn1 = lane + 32 < m ? __ldg(a.v_sq + f + 32 + lane) : INT_MAX;
                knew[lane] = kn0;
                knew[lane + 32] = kn1;
                __syncwarp();
                // owners whose primitive left the list flush and free their slot
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const bool del = key[q] >= 0 && !sorted64_has(knew, key[q]);
                    const unsigned dm = __ballot_sync(0xffffffffu, del);
                    if (dm) {
                        if (qn + __popc(dm) > QCAP) {
                            __syncwarp();
                            drain_queue(A.gacc, wb.queue, qn, lane, gsl, a.C);
                            __syncwarp();
                            qn = 0;
                        }
                        if (del) {
                            float* ent = wb.queue + (qn + __popc(dm & lt)) * QW;
                            ent[0] = __int_as_float(key[q]);
#pragma unroll
                            for (int i = 0; i < 14; ++i) ent[1 + i] = acc[q][i];
                            key[q] = -1;
                        }
                        qn += __popc(dm);
                    }
                }
                // new entries take free slots in rank order
                const bool new0 = lane < m && !sorted64_has(kold, kn0);
                const bool new1 = lane + 32 < m && !sorted64_has(kold, kn1);
                const unsigned nm0 = __ballot_sync(0xffffffffu, new0), nm1 = __ballot_sync(0xffffffffu, new1);
                const int c0 = __popc(nm0), nnew = c0 + __popc(nm1);
                if (nnew) {
                    const unsigned fr0 = __ballot_sync(0xffffffffu, key[0] < 0);
                    const unsigned fr1 = __ballot_sync(0xffffffffu, key[1] < 0);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int rk = (q == 0) ? __popc(fr0 & lt) : __popc(fr0) + __popc(fr1 & lt);
                        const bool want = key[q] < 0 && rk < nnew;
                        int src = lane;
                        bool hi = false;
                        if (want) {
                            if (rk < c0) src = __fns(nm0, 0, rk + 1);
                            else { src = __fns(nm1, 0, rk - c0 + 1); hi = true; }
                        }
                        const int va = __shfl_sync(0xffffffffu, kn0, src);
                        const int vb = __shfl_sync(0xffffffffu, kn1, src);
                        if (want) {
                            key[q] = hi ? vb : va;
#pragma unroll
                            for (int i = 0; i < 14; ++i) acc[q][i] = 0.f;
                            cdk[q] = logit_dot<CP>(a.lpad, key[q], gSr);
                        }
                    }
                }
                int* tmp = kold;
                kold = knew;
                knew = tmp;
                if (j == Le) break;
                // each owner evaluates its pair with sample j
                const bool any1 = __any_sync(0xffffffffu, key[1] >= 0);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (q == 1 && !any1) break;
                    if (key[q] >= 0) {
                        const BwdPrim P = load_bwd(a.rec, a.aux, key[q]);
                        float gg12[12];
                        const float po = occupancy_grad(P, x, gg12);
                        if (po != 0.f) {
                            const float gf = -po * fmaf(G, P.f.sigma, w * cdk[q]);
#pragma unroll
                            for (int i = 0; i < 12; ++i) acc[q][i] = fmaf(gf, gg12[i], acc[q][i]);
                            acc[q][12] = fmaf(G, po, acc[q][12]);
                            acc[q][13] = fmaf(w, po, acc[q][13]);
                        }
                    }
                }
                // list entries beyond the owner slots: per-pair atomics
                for (int e = OWN + lane; e < n; e += 32) {
                    const int k = __ldg(a.v_sq + f + e);
                    const BwdPrim P = load_bwd(a.rec, a.aux, k);
                    float gg12[12];
                    const float po = occupancy_grad(P, x, gg12);
                    if (po == 0.f) continue;
                    const float cd = logit_dot<CP>(a.lpad, k, gSr);
                    const float gf = -po * fmaf(G, P.f.sigma, w * cd);
                    float* dst = A.gacc + (size_t)k * GF;
#pragma unroll
                    for (int i = 0; i < 12; ++i) red_add(dst + i, gf * gg12[i]);
                    red_add(dst + 12, G * po);
#pragma unroll
                    for (int c = 0; c < CP; ++c)
                        if (c < a.C) red_add(dst + NGEO + c, w * po * gSr[c]);
                }
                __syncwarp();
            }
            __syncwarp();
            drain_queue(A.gacc, wb.queue, qn, lane, gsl, a.C);
            __syncwarp();
        }
    }
}

// Scatter of the [N, GF] accumulator into the six gradient outputs.
__global__ void k_grad_out(const float* __restrict__ gacc, int n, int C, float* __restrict__ gm, float* __restrict__ gq,
                           float* __restrict__ gs, float* __restrict__ ge, float* __restrict__ go,
                           float* __restrict__ gl) {
    const long long total = (long long)n * GF;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / GF), fld = (int)(i - (long long)k * GF);
        const float v = gacc[i];
        if (fld < 3) gm[3 * k + fld] = v;
        else if (fld < 7) gq[4 * k + fld - 3] = v;
        else if (fld < 10) gs[3 * k + fld - 7] = v;
        else if (fld < 12) ge[2 * k + fld - 10] = v;
        else if (fld == 12) go[k] = v;
        else if (fld - NGEO < C) gl[(size_t)k * C + fld - NGEO] = v;
    }
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
    size_t rec_off, aux_off, lpad_off, gacc_off, ctr_off, total;
};

static RenderWs render_ws(const sq_prims_t* p) {
    RenderWs w;
    const size_t n = (size_t)(p->n > 0 ? p->n : 0);
    const int cp = cpad(p->n_classes);
    w.rec_off = 0;
    w.aux_off = align_up(n * REC4 * sizeof(float4), 256);
    w.lpad_off = align_up(w.aux_off + n * AUX4 * sizeof(float4), 256);
    w.gacc_off = align_up(w.lpad_off + n * cp * sizeof(float), 256);
    w.ctr_off = align_up(w.gacc_off + n * GF * sizeof(float), 256);
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
    if (gacc) *gacc = (float*)(base + w.gacc_off);
    return SQ_OK;
}

template <int CP>
static sq_status_t launch_fwd_cp(const RenderArgs& a, float* depth, float* sem, float* t_final, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward<CP>, FWD_WARPS * 32, 0);
    if (e != cudaSuccess) return cuda_status(e, "k_forward occupancy");
    long long need = (a.R + FWD_WARPS * NG - 1) / (FWD_WARPS * NG);
    long long blocks = (long long)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k_forward<CP><<<(int)blocks, FWD_WARPS * 32, 0, st>>>(a, depth, sem, t_final);
    SQ_CHECK_LAUNCH("k_forward");
    return SQ_OK;
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
                            const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* ws,
                            size_t ws_bytes, cudaStream_t st) {
    RenderArgs a;
    sq_status_t s = setup_render(prims, idx, grid, rays, ws, ws_bytes, st, false, a, nullptr, "sq_render_fwd");
    if (s != SQ_OK) return s;
    if (a.R == 0) return SQ_OK;
    const int cp = cpad(prims->n_classes);
    SQ_DISPATCH_CP(cp, (launch_fwd_cp<CPV>(a, depth, sem, t_final, st)));
}

static int bwd_warps(int L) {
    const size_t per_warp = sizeof(WarpBwd) + (size_t)NG * 3 * L * sizeof(float);
    int nw = (int)((200 * 1024) / per_warp);
    if (nw > 8) nw = 8;
    if (nw < 1) nw = 1;
    return nw;
}

template <int CP>
static sq_status_t launch_bwd_cp(const BwdArgs& A, cudaStream_t st) {
    const int nw = bwd_warps(A.r.L);
    const size_t smem = (size_t)nw * (sizeof(WarpBwd) + (size_t)NG * 3 * A.r.L * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(k_backward<CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, "k_backward smem attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward<CP>, nw * 32, smem);
    if (e != cudaSuccess) return cuda_status(e, "k_backward occupancy");
    long long need = (A.r.R + (long long)nw * NG - 1) / ((long long)nw * NG);
    long long blocks = (long long)sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k_backward<CP><<<(int)blocks, nw * 32, smem, st>>>(A);
    SQ_CHECK_LAUNCH("k_backward");
    return SQ_OK;
}

sq_status_t render_bwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, const float* grad_depth, const float* grad_sem, float* g_means,
                            float* g_quats, float* g_scales, float* g_eps, float* g_opacity, float* g_logits,
                            void* ws, size_t ws_bytes, cudaStream_t st) {
    BwdArgs A;
    float* gacc = nullptr;
    sq_status_t s = setup_render(prims, idx, grid, rays, ws, ws_bytes, st, true, A.r, &gacc, "sq_render_bwd");
    if (s != SQ_OK) return s;
    const int n = prims->n;
    const int C = prims->n_classes;
    if (n == 0) return SQ_OK;
    cudaError_t e = cudaMemsetAsync(gacc, 0, (size_t)n * GF * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "memset gradient accumulator");
    A.grad_depth = grad_depth;
    A.grad_sem = grad_sem;
    A.gacc = gacc;
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
    long long total = (long long)n * GF;
    int blocks = (int)((total + 255) / 256 < 152LL * 16 ? (total + 255) / 256 : 152LL * 16);
    k_grad_out<<<blocks, 256, 0, st>>>(gacc, n, C, g_means, g_quats, g_scales, g_eps, g_opacity, g_logits);
    SQ_CHECK_LAUNCH("k_grad_out");
    return SQ_OK;
}

}  // namespace sqr
