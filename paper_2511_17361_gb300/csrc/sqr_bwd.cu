// sqr_bwd.cu -- backward render (Sec. 3.3.3) on sm_103a.
//
// One warp per ray, samples back to front.  With T_j saved by the forward, the
// back-to-front carry U_j = alpha_{j+1} v_{j+1} + (1 - alpha_{j+1}) U_{j+1} gives
// dL/dalpha_j = T_j (v_j - U_j) (v_j = gD t_j + <gS, s_j>, zero where the alpha
// clamp is active) in the same sweep that evaluates every pair's gradient.
//
// Along a ray the samples listing a given primitive are contiguous (a ray
// crosses a primitive's voxel box once), so each primitive of the current
// sample's list has an owner slot in a lane that accumulates the primitive's
// partial derivatives in registers while it stays in the lists and flushes them
// once when it leaves (queued, then one coalesced 32-wide atomic add).  Owner
// bookkeeping uses the primitives' voxel boxes: an owner leaves when the sample's
// voxel is outside its box; a list entry is new when the previously processed
// sample's voxel is outside its box.  Lists longer than the 64 owner slots are
// evaluated pair by pair.
#include <limits.h>

#include "sqr_render.cuh"

namespace sqr {

namespace {

constexpr int OWN = 64;   // owner slots per warp (two per lane)
constexpr int QCAP = 64;  // pending flushes per warp
constexpr int QW = 16;    // words per pending flush: key, 11 partials, sigma, W, pad

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
__device__ __forceinline__ void slot_eval(const Slot& S, const SceneDesc& a, const float x[3], float& po, float pr[11],
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

template <int CP>
__global__ void __launch_bounds__(MAX_WARPS * 32, 2) k_backward(Batch B) {
    __shared__ WarpBwd smem[MAX_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float* gSs = smem[wid].gs;

    for (;;) {
        int rr = 0;
        if (lane == 0) rr = atomicAdd(B.ctr, 1);
        const long long gr = __shfl_sync(0xffffffffu, rr, 0);
        if (gr >= B.total) break;
        const int si = scene_of(B, gr);
        const SceneDesc& a = B.d[si];
        const long long r = gr - __ldg(B.off + si);
        if (*a.status != SQ_OK) continue;
        const int Le = __ldg(a.save_n + r);
        __syncwarp();
        gSs[lane] = lane < a.C ? __ldg(a.grad_sem + r * a.C + lane) : 0.f;
        __syncwarp();
        float o[3], d[3];
        scene_ray(a, r, o, d);
        const float gD = __ldg(a.grad_depth + r);
        const float* gS = a.grad_sem + r * a.C;
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
                slot_leave(S0, S0.key >= 0 && (gone || !box_has(S0.box, ix, iy, iz)), Q, a.gacc, lane, lt, gsl, a.C,
                           a.aux);
                slot_leave(S1, S1.key >= 0 && (gone || !box_has(S1.box, ix, iy, iz)), Q, a.gacc, lane, lt, gsl, a.C,
                           a.aux);
                if (!gone) {
                    // list entries whose box misses the previous voxel are new owners
                    int kn0 = -1, kn1 = -1;
                    int4 bx0 = make_int4(1, 1, 1, 0), bx1 = make_int4(1, 1, 1, 0);
                    bool new0 = false, new1 = false;
                    if (lane < n) {
                        kn0 = __ldg(a.v_sq + f + lane);
                        bx0 = __ldg(a.boxes + kn0);
                        new0 = pvox < 0 || !box_has(bx0, pvx, piy, piz);
                    }
                    if (lane + 32 < n) {
                        kn1 = __ldg(a.v_sq + f + lane + 32);
                        bx1 = __ldg(a.boxes + kn1);
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
                        queue_make_room(Q, dm, a.gacc, lane, gsl, a.C, a.aux);
                        queue_push(Q, mine, dm, lt, k, v);
                    }
                }
            }
            U = fmaf(alpha, vj, (1.f - alpha) * U);
        }
        __syncwarp();
        drain_queue(a.gacc, Q.q, Q.n, lane, gsl, a.C);
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


}  // namespace

sq_status_t launch_backward(const Batch& B, int cp, const Tuning& tn, cudaStream_t st) {
    if (B.total == 0) return SQ_OK;
    const int warps = tn.bwd_warps;
    if (warps < 1 || warps > MAX_WARPS) {
        set_last_error("backward tuning (warps %d) not supported", warps);
        return SQ_ERR_INVALID_ARG;
    }
    const void* fn = nullptr;
    switch (cp) {
        case 4: fn = (const void*)k_backward<4>; break;
        case 8: fn = (const void*)k_backward<8>; break;
        case 12: fn = (const void*)k_backward<12>; break;
        case 16: fn = (const void*)k_backward<16>; break;
        case 20: fn = (const void*)k_backward<20>; break;
        case 24: fn = (const void*)k_backward<24>; break;
        case 28: fn = (const void*)k_backward<28>; break;
        case 32: fn = (const void*)k_backward<32>; break;
        default:
            set_last_error("n_classes padding %d not supported", cp);
            return SQ_ERR_INVALID_ARG;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, 0);
    if (e != cudaSuccess) return cuda_status(e, "k_backward occupancy");
    const long long need = (B.total + warps - 1) / warps;
    long long blocks = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    Batch arg = B;
    void* args[] = {&arg};
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(warps * 32), args, 0, st);
    if (e != cudaSuccess) return cuda_status(e, "k_backward");
    return SQ_OK;
}

sq_status_t launch_grad_out(const SceneDesc& S, float* gm, float* gq, float* gs, float* ge, float* go, float* gl,
                            cudaStream_t st) {
    if (S.n == 0) return SQ_OK;
    k_grad_out<<<(S.n + 127) / 128, 128, 0, st>>>(S.gacc, S.aux, S.n, S.C, gm, gq, gs, ge, go, gl);
    SQ_CHECK_LAUNCH("k_grad_out");
    return SQ_OK;
}

sq_status_t launch_pack_boxes(const int* ranges, int n, int4* boxes, cudaStream_t st) {
    if (n == 0) return SQ_OK;
    k_pack_boxes<<<(n + 127) / 128, 128, 0, st>>>(ranges, n, boxes);
    SQ_CHECK_LAUNCH("k_pack_boxes");
    return SQ_OK;
}

}  // namespace sqr
