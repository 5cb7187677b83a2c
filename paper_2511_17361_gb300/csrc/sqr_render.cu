// sqr_render.cu -- forward and backward superquadric volume rendering (Sec. 3.3.2,
// 3.3.3) on sm_103a.
//
// Work decomposition (both passes): one warp marches one ray.  The ray's samples
// are taken in chunks of up to 32 consecutive samples (lane i owns sample j0+i)
// whose voxel lists together hold at most PB (sample, primitive) pairs.  The
// chunk's lists are staged from V_sq into shared memory (coalesced), then the
// lanes sweep the flattened pair list 32 pairs at a time: each lane gathers one
// packed primitive record (4 x float4) and evaluates p_o with the SFU; the pair
// values of one sample are summed with a segmented warp reduction.  Compositing
// of the chunk is a warp product-scan of (1 - alpha).  A single sample whose
// list alone exceeds PB is streamed straight from global memory (occupancies
// recomputed instead of buffered).
//
// Backward: phase 1 replays the forward for the ray and keeps, per sample,
// alpha_j, the clamp flag and v_j = gD t_j + <gS, s_j> in shared memory; phase 2
// sweeps back to front (U_j = alpha_{j+1} v_{j+1} + (1 - alpha_{j+1}) U_{j+1},
// dL/dalpha_j = T_j (v_j - U_j)); phase 3 re-walks the pairs, chains dL/dalpha and
// dL/ds_j through Eq. 1-2 to every parameter, and accumulates the per-primitive
// gradients in a shared-memory hash table owned by the CTA (one table for the
// CTA's tile of rays), flushed to global memory with atomics when the tile ends.
#include <math.h>

#include "sqr_common.cuh"

namespace sqr {

namespace {

constexpr int PB = 256;        // pair buffer per warp (pairs per chunk)
constexpr int FWD_WARPS = 8;   // warps (rays in flight) per CTA, forward
constexpr int BWD_WARPS = 8;   // warps per CTA, backward
constexpr int BWD_RAYS_X = 8;  // backward CTA tile: 8 x 4 pixels
constexpr int BWD_RAYS_Y = 4;
constexpr int TABLE_SLOTS = 512;

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
};

struct ChunkSmem {
    int kbuf[PB];
    float pbuf[PB];
    unsigned char sidx[PB];
    float x[3][32];
    float asum[32];
    float aux[32];
    float wbuf[32];
    int lst[32];
    int cnt[32];
    int off[32];
};

__device__ __forceinline__ void ray_of(const RenderArgs& a, long long r, float o[3], float d[3]) {
    long long hw = (long long)a.H * a.W;
    int cam = (int)(r / hw);
    long long pix = r - (long long)cam * hw;
    int v = (int)(pix / a.W), u = (int)(pix - (long long)v * a.W);
    pixel_ray(a.K + 4 * cam, a.c2w + 12 * cam, u, v, o, d);
}

// Sets up the chunk starting at sample j0: per-lane sample voxel, list start and
// count; returns m (samples in the chunk), pc (pairs), heavy (single sample with
// more than PB pairs).  Stages the lists into shared memory unless heavy.
__device__ __forceinline__ void chunk_setup(const RenderArgs& a, ChunkSmem& sm, const float o[3], const float d[3],
                                            int j0, int lane, int& m, int& pc, bool& heavy) {
    const int j = j0 + lane;
    float x[3] = {0.f, 0.f, 0.f};
    int vox = -1;
    if (j < a.L) vox = sample_voxel(a.g, o, d, __ldg(a.t + j), x);
    int n = 0, f = 0;
    if (vox >= 0) {
        n = __ldg(a.v_n + vox);
        f = __ldg(a.v_f + vox);
    }
    int cum = warp_incl_scan(n, lane);
    unsigned ok = __ballot_sync(0xffffffffu, (cum <= PB) && (j < a.L));
    m = __popc(ok);
    if (m == 0) m = 1;
    pc = __shfl_sync(0xffffffffu, cum, m - 1);
    heavy = pc > PB;
    if (lane < m) {
        sm.x[0][lane] = x[0];
        sm.x[1][lane] = x[1];
        sm.x[2][lane] = x[2];
        sm.asum[lane] = 0.f;
        sm.aux[lane] = 0.f;
        sm.lst[lane] = f;
        sm.cnt[lane] = n;
        sm.off[lane] = cum - n;
    }
    __syncwarp();
    if (!heavy) {
        for (int i = 0; i < m; ++i) {
            const int ni = sm.cnt[i], fi = sm.lst[i], oi = sm.off[i];
            for (int l = lane; l < ni; l += 32) {
                sm.kbuf[oi + l] = __ldg(a.v_sq + fi + l);
                sm.sidx[oi + l] = (unsigned char)i;
            }
        }
    }
    __syncwarp();
}

// Segmented (by sample slot) suffix sum across a 32-pair batch; the first lane of
// each segment ends with the segment total.  Pairs are sorted by slot.
__device__ __forceinline__ float seg_sum(float v, int slot, int lane, bool valid) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float y = __shfl_down_sync(0xffffffffu, v, o);
        int sy = __shfl_down_sync(0xffffffffu, slot, o);
        bool vy = __shfl_down_sync(0xffffffffu, valid, o);
        if (lane + o < 32 && vy && sy == slot) v += y;
    }
    return v;
}

__device__ __forceinline__ bool seg_head(int slot, int lane, bool valid) {
    int sp = __shfl_up_sync(0xffffffffu, slot, 1);
    return valid && (lane == 0 || sp != slot);
}

// Front-to-back compositing of the chunk (Eq. 5): lane i < m holds alpha_i.
// Updates T; returns the lane's weight (0 for lanes >= m or past termination) and
// the number of samples composited in this chunk; sets done on termination.
__device__ __forceinline__ float composite(float alpha, int lane, int m, float kappa, float& T, float& Tbefore,
                                           int& used, bool& done) {
    float om = (lane < m) ? 1.f - alpha : 1.f;
    float incl = warp_incl_prod(om, lane);
    float excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 1.f;
    Tbefore = T * excl;
    float w = (lane < m) ? Tbefore * alpha : 0.f;
    used = m;
    if (kappa > 0.f) {
        unsigned stop = __ballot_sync(0xffffffffu, lane < m && T * incl < kappa);
        if (stop) {
            int ls = __ffs(stop) - 1;
            if (lane > ls) w = 0.f;
            used = ls + 1;
            done = true;
            T = T * __shfl_sync(0xffffffffu, incl, ls);
            return w;
        }
    }
    T = T * __shfl_sync(0xffffffffu, incl, 31);
    if (T == 0.f) done = true;  // every later weight is exactly zero
    return w;
}

// ------------------------------------------------------------------ forward
template <int CP>
__global__ void __launch_bounds__(FWD_WARPS * 32) k_forward(RenderArgs a, float* __restrict__ depth,
                                                            float* __restrict__ sem, float* __restrict__ t_final) {
    __shared__ ChunkSmem smem[FWD_WARPS];
    if (*a.status != SQ_OK) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    ChunkSmem& sm = smem[wid];
    const long long nwarps = (long long)gridDim.x * FWD_WARPS;
    const float4* lp4 = reinterpret_cast<const float4*>(a.lpad);

    for (long long r = (long long)blockIdx.x * FWD_WARPS + wid; r < a.R; r += nwarps) {
        float o[3], d[3];
        ray_of(a, r, o, d);
        float T = 1.f, Dp = 0.f;
        float acc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = 0.f;
        bool done = false;
        for (int j0 = 0; j0 < a.L && !done;) {
            int m, pc;
            bool heavy;
            chunk_setup(a, sm, o, d, j0, lane, m, pc, heavy);
            // pass A: occupancies and alpha sums
            for (int b = 0; b < pc; b += 32) {
                const int gi = b + lane;
                const bool valid = gi < pc;
                int slot = 0;
                float v = 0.f;
                if (valid) {
                    int k;
                    if (!heavy) { k = sm.kbuf[gi]; slot = sm.sidx[gi]; }
                    else k = __ldg(a.v_sq + sm.lst[0] + gi);
                    Prim p = load_prim(a.rec, k);
                    float xs[3] = {sm.x[0][slot], sm.x[1][slot], sm.x[2][slot]};
                    float po = occupancy(p, xs);
                    if (!heavy) sm.pbuf[gi] = po;
                    v = po * p.sigma;
                }
                v = seg_sum(v, slot, lane, valid);
                if (seg_head(slot, lane, valid)) sm.asum[slot] += v;
                __syncwarp();
            }
            __syncwarp();
            float alpha = (lane < m) ? fminf(sm.asum[lane], a.alpha_max) : 0.f;
            float Tb;
            int used;
            float w = composite(alpha, lane, m, a.kappa, T, Tb, used, done);
            if (lane < m) Dp += w * __ldg(a.t + j0 + lane);
            sm.wbuf[lane] = w;
            __syncwarp();
            // pass B: semantics, acc += w_j p c_k
            for (int gi = lane; gi < pc; gi += 32) {
                int k, slot = 0;
                float po;
                if (!heavy) {
                    k = sm.kbuf[gi];
                    slot = sm.sidx[gi];
                    po = sm.pbuf[gi];
                } else {
                    k = __ldg(a.v_sq + sm.lst[0] + gi);
                    Prim p = load_prim(a.rec, k);
                    float xs[3] = {sm.x[0][0], sm.x[1][0], sm.x[2][0]};
                    po = occupancy(p, xs);
                }
                float om = sm.wbuf[slot] * po;
                if (om != 0.f) {
                    const float4* cr = lp4 + (size_t)k * (CP / 4);
#pragma unroll
                    for (int q = 0; q < CP / 4; ++q) {
                        float4 cv = __ldg(cr + q);
                        acc[4 * q + 0] = fmaf(om, cv.x, acc[4 * q + 0]);
                        acc[4 * q + 1] = fmaf(om, cv.y, acc[4 * q + 1]);
                        acc[4 * q + 2] = fmaf(om, cv.z, acc[4 * q + 2]);
                        acc[4 * q + 3] = fmaf(om, cv.w, acc[4 * q + 3]);
                    }
                }
            }
            __syncwarp();
            j0 += m;
        }
        float Dsum = warp_sum(Dp);
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = warp_sum(acc[c]);
        if (lane == 0) {
            depth[r] = Dsum;
            if (t_final) t_final[r] = T;
        }
#pragma unroll
        for (int c = 0; c < CP; ++c)
            if (lane == c && c < a.C) sem[r * a.C + c] = acc[c];
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
    float* g_means;
    float* g_quats;
    float* g_scales;
    float* g_eps;
    float* g_opacity;
    float* g_logits;
    int tiles_x, tiles_y;  // CTA tiles per camera
};

template <int CP>
struct BwdShared {
    static constexpr int NF = 13 + CP;
    static constexpr int STRIDE = NF | 1;
    int keys[TABLE_SLOTS];
    float vals[TABLE_SLOTS * STRIDE];
};

__device__ __forceinline__ unsigned hash_slot(int k) { return ((unsigned)k * 2654435761u) >> 23; }  // 9 bits

template <int CP>
__device__ __forceinline__ void flush_field(const BwdArgs& a, int k, int f, float v) {
    if (v == 0.f) return;
    float* dst;
    if (f < 3) dst = a.g_means + 3 * k + f;
    else if (f < 7) dst = a.g_quats + 4 * k + (f - 3);
    else if (f < 10) dst = a.g_scales + 3 * k + (f - 7);
    else if (f < 12) dst = a.g_eps + 2 * k + (f - 10);
    else if (f == 12) dst = a.g_opacity + k;
    else {
        if (f - 13 >= a.r.C) return;
        dst = a.g_logits + (size_t)k * a.r.C + (f - 13);
    }
    red_add(dst, v);
}

template <int CP>
__global__ void __launch_bounds__(BWD_WARPS * 32) k_backward(BwdArgs a) {
    using SH = BwdShared<CP>;
    extern __shared__ __align__(16) unsigned char dyn[];
    SH& tab = *reinterpret_cast<SH*>(dyn);
    ChunkSmem* chunks = reinterpret_cast<ChunkSmem*>(dyn + align16(sizeof(SH)));
    if (*a.r.status != SQ_OK) return;
    const RenderArgs& ra = a.r;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    ChunkSmem& sm = chunks[wid];
    const int L = ra.L;
    float* samp = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(chunks) + BWD_WARPS * sizeof(ChunkSmem)) +
                  (size_t)wid * 3 * L;
    float* sA = samp;          // alpha_j, negated where the clamp is active; reused as w_j
    float* sV = samp + L;      // v_j; reused as G_j = dL/dalpha_j (0 where clamped)
    float* sT = samp + 2 * L;  // T_j (transmittance before sample j)
    const float4* lp4 = reinterpret_cast<const float4*>(ra.lpad);
    const int tiles_per_cam = a.tiles_x * a.tiles_y;
    const int n_tiles = tiles_per_cam * ra.n_cam;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        for (int s = threadIdx.x; s < TABLE_SLOTS; s += blockDim.x) tab.keys[s] = -1;
        for (int s = threadIdx.x; s < TABLE_SLOTS * SH::STRIDE; s += blockDim.x) tab.vals[s] = 0.f;
        __syncthreads();
        const int cam = tile / tiles_per_cam;
        const int tl = tile - cam * tiles_per_cam;
        const int ty = tl / a.tiles_x, tx = tl - ty * a.tiles_x;
        for (int q = wid; q < BWD_RAYS_X * BWD_RAYS_Y; q += BWD_WARPS) {
            const int u = tx * BWD_RAYS_X + (q % BWD_RAYS_X), v = ty * BWD_RAYS_Y + (q / BWD_RAYS_X);
            if (u >= ra.W || v >= ra.H) continue;
            const long long r = ((long long)cam * ra.H + v) * ra.W + u;
            float o[3], d[3];
            pixel_ray(ra.K + 4 * cam, ra.c2w + 12 * cam, u, v, o, d);
            const float gD = __ldg(a.grad_depth + r);
            float gS[CP];
#pragma unroll
            for (int c = 0; c < CP; ++c) gS[c] = c < ra.C ? __ldg(a.grad_sem + r * ra.C + c) : 0.f;

            // ---- phase 1: replay alpha_j and v_j
            float T = 1.f;
            bool done = false;
            int Leff = 0;
            for (int j0 = 0; j0 < L && !done;) {
                int m, pc;
                bool heavy;
                chunk_setup(ra, sm, o, d, j0, lane, m, pc, heavy);
                for (int b = 0; b < pc; b += 32) {
                    const int gi = b + lane;
                    const bool valid = gi < pc;
                    int slot = 0;
                    float va = 0.f, vs = 0.f;
                    if (valid) {
                        int k;
                        if (!heavy) { k = sm.kbuf[gi]; slot = sm.sidx[gi]; }
                        else k = __ldg(ra.v_sq + sm.lst[0] + gi);
                        Prim p = load_prim(ra.rec, k);
                        float xs[3] = {sm.x[0][slot], sm.x[1][slot], sm.x[2][slot]};
                        float po = occupancy(p, xs);
                        const float4* cr = lp4 + (size_t)k * (CP / 4);
                        float cd = 0.f;
#pragma unroll
                        for (int qq = 0; qq < CP / 4; ++qq) {
                            float4 cv = __ldg(cr + qq);
                            cd = fmaf(gS[4 * qq + 0], cv.x, cd);
                            cd = fmaf(gS[4 * qq + 1], cv.y, cd);
                            cd = fmaf(gS[4 * qq + 2], cv.z, cd);
                            cd = fmaf(gS[4 * qq + 3], cv.w, cd);
                        }
                        va = po * p.sigma;
                        vs = po * cd;
                    }
                    va = seg_sum(va, slot, lane, valid);
                    vs = seg_sum(vs, slot, lane, valid);
                    if (seg_head(slot, lane, valid)) {
                        sm.asum[slot] += va;
                        sm.aux[slot] += vs;
                    }
                    __syncwarp();
                }
                __syncwarp();
                float raw = (lane < m) ? sm.asum[lane] : 0.f;
                float alpha = fminf(raw, ra.alpha_max);
                float Tb;
                int used;
                composite(alpha, lane, m, ra.kappa, T, Tb, used, done);
                if (lane < used) {
                    const int j = j0 + lane;
                    // alpha_max > 0, so a clamped alpha is positive and its sign is free
                    sA[j] = (raw > ra.alpha_max) ? -alpha : alpha;
                    sV[j] = fmaf(gD, __ldg(ra.t + j), sm.aux[lane]);
                    sT[j] = Tb;
                }
                __syncwarp();
                j0 += used;
                Leff = j0;
            }
            // ---- phase 2: back-to-front sweep (lane 0), G_j and w_j
            if (lane == 0) {
                float U = 0.f;
                for (int j = Leff - 1; j >= 0; --j) {
                    float sa = sA[j], vj = sV[j], Tj = sT[j];
                    bool clamped = sa < 0.f;
                    float al = fabsf(sa);
                    float G = clamped ? 0.f : Tj * (vj - U);
                    U = fmaf(al, vj, (1.f - al) * U);
                    sV[j] = G;
                    sA[j] = Tj * al;
                }
            }
            __syncwarp();
            // ---- phase 3: per-pair gradients into the CTA table
            for (int j0 = 0; j0 < Leff;) {
                int m, pc;
                bool heavy;
                chunk_setup(ra, sm, o, d, j0, lane, m, pc, heavy);
                if (j0 + m > Leff) m = Leff - j0;  // pairs of samples past termination are skipped below
                for (int gi = lane; gi < pc; gi += 32) {
                    int k, slot = 0;
                    if (!heavy) { k = sm.kbuf[gi]; slot = sm.sidx[gi]; }
                    else k = __ldg(ra.v_sq + sm.lst[0] + gi);
                    if (slot >= m) continue;
                    const int j = j0 + slot;
                    const float G = sV[j], w = sA[j];
                    if (G == 0.f && w == 0.f) continue;
                    BwdPrim P = load_bwd(ra.rec, ra.aux, k);
                    float xs[3] = {sm.x[0][slot], sm.x[1][slot], sm.x[2][slot]};
                    float gg[12];
                    float po = occupancy_grad(P, xs, gg);
                    if (po == 0.f) continue;
                    const float4* cr = lp4 + (size_t)k * (CP / 4);
                    float cv[CP];
                    float cd = 0.f;
#pragma unroll
                    for (int qq = 0; qq < CP / 4; ++qq) {
                        float4 c4 = __ldg(cr + qq);
                        cv[4 * qq + 0] = c4.x; cv[4 * qq + 1] = c4.y; cv[4 * qq + 2] = c4.z; cv[4 * qq + 3] = c4.w;
                        cd = fmaf(gS[4 * qq + 0], c4.x, cd);
                        cd = fmaf(gS[4 * qq + 1], c4.y, cd);
                        cd = fmaf(gS[4 * qq + 2], c4.z, cd);
                        cd = fmaf(gS[4 * qq + 3], c4.w, cd);
                    }
                    const float dLdp = fmaf(G, P.f.sigma, w * cd);
                    const float gf = -po * dLdp;
                    const float wp = w * po;
                    // find / claim the table slot of primitive k
                    unsigned h = hash_slot(k) & (TABLE_SLOTS - 1);
                    int slotk = -1;
                    for (int probe = 0; probe < TABLE_SLOTS; ++probe) {
                        int key = tab.keys[h];
                        if (key == k) { slotk = (int)h; break; }
                        if (key == -1) {
                            int old = atomicCAS(&tab.keys[h], -1, k);
                            if (old == -1 || old == k) { slotk = (int)h; break; }
                        }
                        h = (h + 1) & (TABLE_SLOTS - 1);
                    }
                    if (slotk >= 0) {
                        float* dst = tab.vals + slotk * SH::STRIDE;
#pragma unroll
                        for (int f = 0; f < 12; ++f) atomicAdd(dst + f, gf * gg[f]);
                        atomicAdd(dst + 12, G * po);
#pragma unroll
                        for (int c = 0; c < CP; ++c)
                            if (c < ra.C) atomicAdd(dst + 13 + c, wp * gS[c]);
                    } else {
#pragma unroll
                        for (int f = 0; f < 12; ++f) flush_field<CP>(a, k, f, gf * gg[f]);
                        flush_field<CP>(a, k, 12, G * po);
#pragma unroll
                        for (int c = 0; c < CP; ++c) flush_field<CP>(a, k, 13 + c, wp * gS[c]);
                    }
                }
                __syncwarp();
                j0 += m;
            }
        }
        __syncthreads();
        // flush the tile's table
        for (int e = threadIdx.x; e < TABLE_SLOTS * SH::NF; e += blockDim.x) {
            int s = e / SH::NF, f = e - s * SH::NF;
            int k = tab.keys[s];
            if (k >= 0) flush_field<CP>(a, k, f, tab.vals[s * SH::STRIDE + f]);
        }
        __syncthreads();
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

// ------------------------------------------------------------------ host side
sq_status_t launch_pack(const sq_prims_t* prims, float4* rec, float4* aux, float* lpad, int cp, cudaStream_t st) {
    if (prims->n == 0) return SQ_OK;
    k_pack<<<(prims->n + 127) / 128, 128, 0, st>>>(*prims, rec, aux, lpad, cp);
    SQ_CHECK_LAUNCH("k_pack");
    return SQ_OK;
}

struct RenderWs {
    size_t rec_off, aux_off, lpad_off, total;
};

static RenderWs render_ws(const sq_prims_t* p) {
    RenderWs w;
    const size_t n = (size_t)(p->n > 0 ? p->n : 0);
    const int cp = cpad(p->n_classes);
    w.rec_off = 0;
    w.aux_off = align_up(n * REC4 * sizeof(float4), 256);
    w.lpad_off = align_up(w.aux_off + n * AUX4 * sizeof(float4), 256);
    w.total = align_up(w.lpad_off + n * cp * sizeof(float), 256);
    if (w.total == 0) w.total = 256;
    return w;
}

size_t render_workspace_size(const sq_prims_t* p) { return render_ws(p).total; }

static sq_status_t setup_render(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                                const sq_rays_t* rays, void* ws, size_t ws_bytes, cudaStream_t st, bool need_aux,
                                RenderArgs& a, const char* who) {
    RenderWs w = render_ws(prims);
    if (ws == nullptr || ws_bytes < w.total) {
        set_last_error("%s: workspace of %zu bytes given, %zu needed", who, ws_bytes, w.total);
        return SQ_ERR_INVALID_ARG;
    }
    char* base = (char*)ws;
    float4* rec = (float4*)(base + w.rec_off);
    float4* aux = need_aux ? (float4*)(base + w.aux_off) : nullptr;
    float* lpad = (float*)(base + w.lpad_off);
    const int cp = cpad(prims->n_classes);
    sq_status_t s = launch_pack(prims, rec, aux, lpad, cp, st);
    if (s != SQ_OK) return s;
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
    a.R = (long long)rays->n_cam * rays->H * rays->W;
    a.kappa = rays->kappa;
    a.alpha_max = rays->alpha_max;
    return SQ_OK;
}

template <int CP>
static sq_status_t launch_fwd_cp(const RenderArgs& a, float* depth, float* sem, float* t_final, cudaStream_t st) {
    long long want = (a.R + FWD_WARPS - 1) / FWD_WARPS;
    int blocks = (int)(want < 152LL * 32 ? want : 152LL * 32);
    if (blocks < 1) blocks = 1;
    k_forward<CP><<<blocks, FWD_WARPS * 32, 0, st>>>(a, depth, sem, t_final);
    SQ_CHECK_LAUNCH("k_forward");
    return SQ_OK;
}

#define SQ_DISPATCH_CP(cp, CALL)        \
    switch (cp) {                       \
        case 4: { constexpr int CPV = 4; return CALL; }   \
        case 8: { constexpr int CPV = 8; return CALL; }   \
        case 12: { constexpr int CPV = 12; return CALL; } \
        case 16: { constexpr int CPV = 16; return CALL; } \
        case 20: { constexpr int CPV = 20; return CALL; } \
        case 24: { constexpr int CPV = 24; return CALL; } \
        case 28: { constexpr int CPV = 28; return CALL; } \
        case 32: { constexpr int CPV = 32; return CALL; } \
        default: return SQ_ERR_INVALID_ARG;                \
    }

sq_status_t render_fwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* ws,
                            size_t ws_bytes, cudaStream_t st) {
    RenderArgs a;
    sq_status_t s = setup_render(prims, idx, grid, rays, ws, ws_bytes, st, false, a, "sq_render_fwd");
    if (s != SQ_OK) return s;
    if (a.R == 0) return SQ_OK;
    const int cp = cpad(prims->n_classes);
    SQ_DISPATCH_CP(cp, (launch_fwd_cp<CPV>(a, depth, sem, t_final, st)));
}

template <int CP>
static size_t bwd_smem_bytes(int L) {
    return align16(sizeof(BwdShared<CP>)) + BWD_WARPS * sizeof(ChunkSmem) + (size_t)BWD_WARPS * 3 * L * sizeof(float);
}

template <int CP>
static sq_status_t launch_bwd_cp(const BwdArgs& a, cudaStream_t st) {
    size_t smem = bwd_smem_bytes<CP>(a.r.L);
    cudaError_t e = cudaFuncSetAttribute(k_backward<CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, "k_backward smem attribute");
    int n_tiles = a.tiles_x * a.tiles_y * a.r.n_cam;
    k_backward<CP><<<n_tiles, BWD_WARPS * 32, smem, st>>>(a);
    SQ_CHECK_LAUNCH("k_backward");
    return SQ_OK;
}

sq_status_t render_bwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, const float* grad_depth, const float* grad_sem, float* g_means,
                            float* g_quats, float* g_scales, float* g_eps, float* g_opacity, float* g_logits,
                            void* ws, size_t ws_bytes, cudaStream_t st) {
    BwdArgs a;
    sq_status_t s = setup_render(prims, idx, grid, rays, ws, ws_bytes, st, true, a.r, "sq_render_bwd");
    if (s != SQ_OK) return s;
    const size_t n = (size_t)prims->n;
    const int C = prims->n_classes;
    struct { float* p; size_t count; } outs[6] = {{g_means, 3 * n}, {g_quats, 4 * n}, {g_scales, 3 * n},
                                                {g_eps, 2 * n},   {g_opacity, n},    {g_logits, C * n}};
    for (auto& o : outs) {
        if (o.count == 0) continue;
        cudaError_t e = cudaMemsetAsync(o.p, 0, o.count * sizeof(float), st);
        if (e != cudaSuccess) return cuda_status(e, "memset gradients");
    }
    if (a.r.R == 0 || n == 0) return SQ_OK;
    a.grad_depth = grad_depth;
    a.grad_sem = grad_sem;
    a.g_means = g_means;
    a.g_quats = g_quats;
    a.g_scales = g_scales;
    a.g_eps = g_eps;
    a.g_opacity = g_opacity;
    a.g_logits = g_logits;
    a.tiles_x = (rays->W + BWD_RAYS_X - 1) / BWD_RAYS_X;
    a.tiles_y = (rays->H + BWD_RAYS_Y - 1) / BWD_RAYS_Y;
    const int cp = cpad(C);
    SQ_DISPATCH_CP(cp, (launch_bwd_cp<CPV>(a, st)));
}

}  // namespace sqr
