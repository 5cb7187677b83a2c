// sqr_fwd.cu -- forward render (Sec. 3.3.2, Eq. 2, 4-6) on sm_103a.
//
// A warp marches 32/GS rays at a time, GS lanes per ray, one lane per sample.
// Each lane sums its own sample's voxel list (Sec. 3.3.1), so the sums of Eq. 4
// (alpha = sum p sigma, s = sum p c) stay in the lane's registers; the GS lanes
// walk their lists together in ascending primitive order, so that a record that
// several neighbouring samples need is loaded once for all of them; compositing
// (Eq. 5-6) of a group's GS samples is a GS-lane product scan of (1 - alpha).
// Rays of all scenes of the batch are handed out by one global counter, so a
// lane group whose ray ends early takes the next ray, from whichever scene.
// For the backward the forward saves, per composited sample, T_j, alpha_j (sign
// marking the clamp) and s_j, in pages of SAVE_PS samples handed out as rays
// advance (only composited chunks take memory), and per ray the number of
// composited samples.
#include <limits.h>

#include "sqr_render.cuh"

namespace sqr {

namespace {

template <int GS>
__device__ __forceinline__ float group_incl_prod(float v, int s) {
#pragma unroll
    for (int o = 1; o < GS; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, v, o, GS);
        if (s >= o) v *= y;
    }
    return v;
}

// Compositing (Eq. 5) of a group's GS consecutive samples.  Lane s holds alpha
// (0 for lanes past L or outside the grid).  Returns w = T_before * alpha (0 past
// an early termination) and T_before; advances T (uniform in the group); `stop`
// when kappa > 0 ends the ray inside this chunk, `used` = samples composited.
template <int GS>
__device__ __forceinline__ float group_composite(float alpha, int s, int gbase, float kappa, float& T, float& Tb,
                                                 bool valid, int& used, bool& stop) {
    const float incl = group_incl_prod<GS>(1.f - alpha, s);
    float excl = __shfl_up_sync(0xffffffffu, incl, 1, GS);
    if (s == 0) excl = 1.f;
    Tb = T * excl;
    float w = Tb * alpha;
    used = GS;
    stop = false;
    const unsigned gmask = (GS == 32) ? 0xffffffffu : ((1u << GS) - 1u);
    const unsigned kill = __ballot_sync(0xffffffffu, valid && kappa > 0.f && T * incl < kappa);
    const unsigned gk = (kill >> gbase) & gmask;
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

template <int CP, int GS, bool TILED>
__global__ void __launch_bounds__(MAX_WARPS * 32) k_forward(Batch B) {
    static_assert(GS % SAVE_PS == 0 || SAVE_PS % GS == 0, "chunks and pages of the saved state nest");
    const int lane = threadIdx.x & 31;
    const int s = lane & (GS - 1), gbase = lane & ~(GS - 1);
    const unsigned gmask = (GS == 32) ? 0xffffffffu : ((1u << GS) - 1u);

    // draw the group's first ray: the group takes B.ray_tile consecutive rays from
    // the work counter at a time (a tile of neighbouring pixels) and marches them in turn
    const int rt = TILED ? B.ray_tile : 1;
    int gn = 0;
    if (s == 0) gn = atomicAdd(B.ctr, rt);
    long long gr = __shfl_sync(0xffffffffu, gn, gbase);
    long long tend = gr + rt;  // end of the group's tile
    int si = 0;
    long long r = 0;
    bool live = gr < B.total;
    if (live) {
        si = scene_of(B, gr);
        r = gr - __ldg(B.off + si);
        if (*B.d[si].status != SQ_OK) live = false;
    }
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f};
    if (live) scene_ray(B.d[si], r, o, d);
    float T = 1.f, Dp = 0.f;
    int j0 = 0, used_total = 0;
    int last_pg = -1;  // the ray's most recent page of saved state (the same in the lane group)
    bool seen_inside = false;
    float acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = 0.f;

    while (__any_sync(0xffffffffu, gr < B.total)) {
        const SceneDesc& S = B.d[si];
        // scene constants of this group's ray, kept in registers for the list walk
        const int L = S.L;
        const float4* __restrict__ rec = S.rec;
        const float4* __restrict__ lp4 = reinterpret_cast<const float4*>(S.lpad);
        const int* __restrict__ v_sq = S.v_sq;
        const int j = j0 + s;
        const bool valid = live && j < L;
        // Pages of the saved state for this chunk: the counter update is issued here
        // and its result read after the list walk, which hides its latency.  In a
        // launch over one scene the groups' requests (0, 1 or 2 pages each) are
        // combined into one update per warp by ballots; over several scenes each
        // group asks its own buffer's counter.
        const int fp = (j0 + SAVE_PS - 1) / SAVE_PS;  // the pages that start in this chunk: fp .. fp + cntg - 1
        const int cntg = (live && S.save_TA != nullptr) ? max(0, (min(j0 + GS, L) - 1) / SAVE_PS - fp + 1) : 0;
        const int cnt = s == 0 ? cntg : 0;
        static_assert(GS <= 2 * SAVE_PS, "at most two pages per chunk");
        const unsigned b1 = __ballot_sync(0xffffffffu, cnt >= 1), b2 = __ballot_sync(0xffffffffu, cnt >= 2);
        const unsigned lt = (1u << lane) - 1u;
        const int before = __popc(b1 & lt) + __popc(b2 & lt);  // pages of the lower groups
        unsigned long long pbase = 0;
        if (B.n == 1) {
            if (lane == 0 && b1 != 0u) pbase = atomicAdd(S.save_ctr, (unsigned long long)(__popc(b1) + __popc(b2)));
        } else if (cnt > 0) {
            pbase = atomicAdd(S.save_ctr, (unsigned long long)cnt);
        }
        float x[3] = {0.f, 0.f, 0.f};
        int vox = -1;
        float tj = 0.f;
        if (valid) {
            tj = __ldg(S.t + j);
            const GridC g = S.g;
            vox = sample_voxel(g, o, d, tj, x);
        }
        int n = 0, f = 0;
        if (vox >= 0) {
            n = __ldg(S.v_n + vox);
            f = __ldg(S.v_f + vox);
            if (n > 0 && !SQ_BOUND(f >= 0 && (long long)f + n <= S.v_cap, 1)) n = 0;
        }
        float asum = 0.f;
        float sacc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) sacc[c] = 0.f;
        // Merge-walk of the group's lists (each ascending in primitive id): every
        // step takes the smallest pending id of the group, loads its record once
        // for the group (one address, a broadcast) and adds it to the samples whose
        // list holds it.  Each sample still sums its list in ascending id order.
        int e = 0;
        int head = n > 0 ? __ldg(v_sq + f) : INT_MAX;
        int head2 = n > 1 ? __ldg(v_sq + f + 1) : INT_MAX;
        int head3 = n > 2 ? __ldg(v_sq + f + 2) : INT_MAX;  // list look-ahead of two
        int kmin = head;
#pragma unroll
        for (int o2 = GS / 2; o2 > 0; o2 >>= 1) kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o2, GS));
        Prim p;  // the group's record, loaded one step ahead
        if (kmin != INT_MAX && SQ_BOUND((unsigned)kmin < (unsigned)S.n, 2)) p = load_prim(rec, kmin);
        while (__any_sync(0xffffffffu, kmin != INT_MAX)) {
            // the group's next id is known before this step's work: its record loads overlap the math
            int knext = head == kmin ? head2 : head;
#pragma unroll
            for (int o2 = GS / 2; o2 > 0; o2 >>= 1) knext = min(knext, __shfl_xor_sync(0xffffffffu, knext, o2, GS));
            Prim pn;
            if (knext != INT_MAX && SQ_BOUND((unsigned)knext < (unsigned)S.n, 2)) pn = load_prim(rec, knext);
            if (kmin != INT_MAX) {
                // (a listed id that is not a primitive is skipped, its list still advances)
                const bool idok = SQ_BOUND((unsigned)kmin < (unsigned)S.n, 2);
                const float4* cr = lp4 + (size_t)(idok ? kmin : 0) * (CP / 4);
                float4 cv[CP / 4];
#pragma unroll
                for (int q = 0; q < CP / 4; ++q) cv[q] = idok ? __ldg(cr + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (head == kmin) {
                    if (idok) {
                        const float po = occupancy(p, x);
                        asum = fmaf(po, p.sigma, asum);
#pragma unroll
                        for (int q = 0; q < CP / 4; ++q) {
                            sacc[4 * q + 0] = fmaf(po, cv[q].x, sacc[4 * q + 0]);
                            sacc[4 * q + 1] = fmaf(po, cv[q].y, sacc[4 * q + 1]);
                            sacc[4 * q + 2] = fmaf(po, cv[q].z, sacc[4 * q + 2]);
                            sacc[4 * q + 3] = fmaf(po, cv[q].w, sacc[4 * q + 3]);
                        }
                    }
                    ++e;
                    head = head2;
                    head2 = head3;
                    head3 = e + 2 < n ? __ldg(v_sq + f + e + 2) : INT_MAX;
                }
            }
            kmin = knext;
            p = pn;
        }
        const float alpha = valid ? fminf(asum, S.alpha_max) : 0.f;
        float Tb;
        int used;
        bool stop;
        const float w = group_composite<GS>(alpha, s, gbase, S.kappa, T, Tb, valid, used, stop);
        // the chunk's pages: the group's first page, a page table entry per page; a
        // group past the buffer's capacity marks the overflow and saves nothing (its
        // rays' backward then does no work)
        int pg;
        {
            const unsigned long long wb = __shfl_sync(0xffffffffu, pbase, 0);
            int first = -1;
            if (cnt > 0) {
                const long long f = B.n == 1 ? (long long)wb + before : (long long)pbase;
                const bool fits = f + cnt <= S.save_cap;
                if (!fits) atomicExch(S.save_status, (int)SQ_ERR_CAPACITY);
                for (int i = 0; i < cnt; ++i) S.save_page[r * S.save_np + fp + i] = fits ? (int)(f + i) : -1;
                first = fits ? (int)f : -1;
            }
            first = __shfl_sync(0xffffffffu, first, gbase);
            // a sample in a page begun by an earlier chunk goes to the ray's last page
            const int pi = j / SAVE_PS;
            pg = pi >= fp ? (first >= 0 ? first + (pi - fp) : -1) : last_pg;
            if (cntg > 0) last_pg = first >= 0 ? first + cntg - 1 : -1;
        }
        if (valid) {
            if (s < used && pg >= 0) {
                const long long sj = (long long)pg * SAVE_PS + (j % SAVE_PS);
                S.save_TA[sj] = make_float2(Tb, asum > S.alpha_max ? -alpha : alpha);
                float4* sv = S.save_S + sj * (CP / 4);
#pragma unroll
                for (int q = 0; q < CP / 4; ++q)
                    sv[q] = make_float4(sacc[4 * q], sacc[4 * q + 1], sacc[4 * q + 2], sacc[4 * q + 3]);
            }
            Dp = fmaf(w, tj, Dp);
#pragma unroll
            for (int c = 0; c < CP; ++c) acc[c] = fmaf(w, sacc[c], acc[c]);
        }
        // t is non-decreasing, so a chunk fully outside the grid after an inside
        // one means the ray has left the grid for good
        const unsigned ins = (__ballot_sync(0xffffffffu, vox >= 0) >> gbase) & gmask;
        const bool left = seen_inside && ins == 0u;
        seen_inside = seen_inside || ins != 0u;
        if (live) used_total = min(j0 + used, L);
        j0 += GS;
        // a ray ends at L, on early termination, once T is exactly 0 (every later
        // weight is 0), or when it has left the grid
        const bool fin = (gr < B.total) && (!live || j0 >= L || stop || T == 0.f || left);
        if (__any_sync(0xffffffffu, fin)) {
            float Dsum = Dp;
#pragma unroll
            for (int o2 = GS / 2; o2 > 0; o2 >>= 1) Dsum += __shfl_xor_sync(0xffffffffu, Dsum, o2, GS);
#pragma unroll
            for (int c = 0; c < CP; ++c) {
                float v = acc[c];
#pragma unroll
                for (int o2 = GS / 2; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2, GS);
                if (fin && live && (c % GS) == s && c < S.C) S.sem[r * S.C + c] = v;
            }
            if (fin && live && s == 0) {
                S.depth[r] = Dsum;
                if (S.t_final) S.t_final[r] = T;
                if (S.save_n) S.save_n[r] = used_total;
            }
            int nr = 0;
            const bool refill = fin && (!TILED || gr + 1 >= tend);
            if (refill && s == 0) nr = atomicAdd(B.ctr, rt);
            nr = __shfl_sync(0xffffffffu, nr, gbase);
            if (fin) {
                gr = refill ? (long long)nr : gr + 1;
                if (TILED && refill) tend = gr + rt;
                live = gr < B.total;
                if (live) {
                    si = scene_of(B, gr);
                    r = gr - __ldg(B.off + si);
                    if (*B.d[si].status != SQ_OK) live = false;
                }
                if (live) scene_ray(B.d[si], r, o, d);
                T = 1.f;
                Dp = 0.f;
                j0 = 0;
                used_total = 0;
                last_pg = -1;
                seen_inside = false;
#pragma unroll
                for (int c = 0; c < CP; ++c) acc[c] = 0.f;
            }
        }
    }
}

template <int CP, int GS, bool TILED>
sq_status_t launch_cp_gs_t(const Batch& B, int warps, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward<CP, GS, TILED>, warps * 32, 0);
    if (e != cudaSuccess) return cuda_status(e, "k_forward occupancy");
    const long long per_block = (long long)warps * (32 / GS);
    const long long need = (B.total + per_block - 1) / per_block;
    long long blocks = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    SQ_LAUNCH("k_forward", st, k_forward<CP, GS, TILED><<<(int)blocks, warps * 32, 0, st>>>(B));
    return SQ_OK;
}

// Ray tiles of more than one ray take a separate instance, so that the default
// (one ray per fetch) is compiled without the tile bookkeeping.
template <int CP, int GS>
sq_status_t launch_cp_gs(const Batch& B, int warps, cudaStream_t st) {
    return B.ray_tile > 1 ? launch_cp_gs_t<CP, GS, true>(B, warps, st) : launch_cp_gs_t<CP, GS, false>(B, warps, st);
}

template <int CP>
sq_status_t launch_cp(const Batch& B, const Tuning& tn, cudaStream_t st) {
    if (tn.fwd_lanes == 16) return launch_cp_gs<CP, 16>(B, tn.fwd_warps, st);
    if (tn.fwd_lanes == 8) return launch_cp_gs<CP, 8>(B, tn.fwd_warps, st);
    return launch_cp_gs<CP, 4>(B, tn.fwd_warps, st);
}

}  // namespace

sq_status_t launch_forward(const Batch& B, int cp, const Tuning& tn, cudaStream_t st) {
    if (B.total == 0) return SQ_OK;
    if (tn.fwd_warps < 1 || tn.fwd_warps > MAX_WARPS || (tn.fwd_lanes != 4 && tn.fwd_lanes != 8 && tn.fwd_lanes != 16)) {
        set_last_error("forward tuning (lanes %d, warps %d) not supported", tn.fwd_lanes, tn.fwd_warps);
        return SQ_ERR_INVALID_ARG;
    }
    switch (cp) {
        case 4: return launch_cp<4>(B, tn, st);
        case 8: return launch_cp<8>(B, tn, st);
        case 12: return launch_cp<12>(B, tn, st);
        case 16: return launch_cp<16>(B, tn, st);
        case 20: return launch_cp<20>(B, tn, st);
        case 24: return launch_cp<24>(B, tn, st);
        case 28: return launch_cp<28>(B, tn, st);
        case 32: return launch_cp<32>(B, tn, st);
    }
    set_last_error("n_classes padding %d not supported", cp);
    return SQ_ERR_INVALID_ARG;
}

#ifdef SQR_CHECK
unsigned check_take_fwd() { return check_take(); }
#endif

}  // namespace sqr
