// sqr_bwd.cu -- backward render (Sec. 3.3.3) on sm_103a, in two launches.
//
// k_bwd_sweep (one warp per ray, samples back to front): from the forward's saved
// alpha_j, s_j and T_j it forms v_j = gD t_j + <gS, s_j> and the carry
// U_j = alpha_{j+1} v_{j+1} + (1 - alpha_{j+1}) U_{j+1} (a 32-lane suffix scan of
// affine maps per chunk of 32 samples), and writes dL/dalpha_j = T_j (v_j - U_j)
// (zero where the alpha clamp is active) and w_j = T_j alpha_j per sample.
//
// k_backward (one warp per bundle of RB rays): along a ray the samples whose lists
// hold a given primitive are consecutive (the voxel coordinates of the samples are
// monotone in t and the primitive is listed in exactly the voxels of its box), so
// every (ray, primitive) pair is one run of samples.  Per bundle the warp builds a
// sample table in shared memory (point, voxel, list, dL/dalpha_j, w_j), lists the
// runs that start at each sample (list entries whose voxel range misses the
// previous sample's voxel, read from the index's range-boundary flags when it has
// them), finds each run's end by a binary search, and then every lane
// walks runs on its own: it holds the primitive's record in registers, evaluates
// dp_o/d(params) at the run's samples (two per step), weights them by
// dL/dp_o = G_j sigma + w_j <gS, c>, sums in registers and flushes once per run
// (queued in shared memory, then coalesced atomic adds of raw partial sums).
// Idle lanes take the next listed runs together.  k_grad_out turns the sums into
// parameter gradients.
#include "sqr_pair.cuh"
#include "sqr_render.cuh"

namespace sqr {

namespace {

constexpr int RB = 2;      // rays per bundle
constexpr int TCAP = 256;  // runs listed per pass
constexpr int RTH = 4;     // idle lanes that trigger a refill while others still walk
constexpr int LU = 8;      // 32-entry batches whose loads the run listing issues together
constexpr int RU = 4;      // listed runs per lane whose loads the per-run pass issues together
constexpr int NS = 2;      // samples of a run a lane evaluates per walker step
constexpr int QCAP = 32;   // pending flushes per warp
constexpr int QW = 16;     // words per flush: 11 partials, sigma, W, primitive, ray slot, pad
static_assert(QCAP >= 32, "one walker step can end a run in every lane");
static_assert(TCAP >= 32 && TCAP % 32 == 0, "the listing appends up to 32 runs at a time");

__global__ void k_pack_boxes(const int* __restrict__ ranges, int n, int4* __restrict__ boxes) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int* r = ranges + 6 * k;
    int v[3];
    const bool empty = r[1] < r[0] || r[3] < r[2] || r[5] < r[4];
    for (int a = 0; a < 3; ++a) v[a] = empty ? 1 : (r[2 * a] | (r[2 * a + 1] << 16));
    boxes[k] = make_int4(v[0], v[1], v[2], 0);
}


// Packed inclusive box test; an empty box is stored as lo = 1, hi = 0.  pv holds
// a sample's voxel as (ix | iy << 16, iz | extra << 16), pv.y = -1 outside the grid.
__device__ __forceinline__ bool box_has(const int4 b, int2 pv) {
    if (pv.y < 0) return false;
    const unsigned bx = (unsigned)b.x, by = (unsigned)b.y, bz = (unsigned)b.z, px = (unsigned)pv.x;
    const unsigned ix = px & 0xffffu, iy = px >> 16, iz = (unsigned)pv.y & 0xffffu;
    return ix >= (bx & 0xffffu) && ix <= (bx >> 16) && iy >= (by & 0xffffu) && iy <= (by >> 16) &&
           iz >= (bz & 0xffffu) && iz <= (bz >> 16);
}

// <gS, c_k> with gS staged in shared memory (zero-padded to 32).
template <int CP>
__device__ __forceinline__ float logit_dot(const float* __restrict__ lpad, int k, const float* gs) {
    const float4* cr = reinterpret_cast<const float4*>(lpad) + (size_t)k * (CP / 4);
    float cd = 0.f;
#pragma unroll
    for (int q = 0; q < CP / 4; ++q) {
        const float4 c4 = __ldg(cr + q);
        cd = fmaf(gs[4 * q + 0], c4.x, cd);
        cd = fmaf(gs[4 * q + 1], c4.y, cd);
        cd = fmaf(gs[4 * q + 2], c4.z, cd);
        cd = fmaf(gs[4 * q + 3], c4.w, cd);
    }
    return cd;
}

// Vector atomic add of four floats (16-byte aligned address).
__device__ __forceinline__ void red_add4(float* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Writes the warp's pending flushes into the accumulator of raw partial sums,
// four entries per pass (two when n_classes > 20): lane (e, i) adds float4 i of
// entry e's row.  A queue
// entry holds the 12 summed partials (gx 3, tau 3, u df/du 3, eps 2, sigma 1), W,
// the primitive and the ray slot; row fields 12.. are the logit gradients W gS_c
// of that ray (gS of the bundle's rays in gsb, zero-padded to 32).
__device__ __forceinline__ void drain_queue(float* __restrict__ gacc, const float* __restrict__ q, int qn, int lane,
                                            const float* __restrict__ gsb, int C) {
    const int sh = NRAW + C > 32 ? 4 : 3;  // log2 of the lanes per entry
    const int sub = lane >> sh, i = lane & ((1 << sh) - 1);
    const bool used = 4 * i < NRAW + C;
    for (int e0 = 0; e0 < qn; e0 += 32 >> sh) {
        const int e = e0 + sub;
        if (e < qn && used) {
            const float* ent = q + e * QW;
            const int k = __float_as_int(ent[13]);
            float4 v;
            if (i < 3) {
                v = *reinterpret_cast<const float4*>(ent + 4 * i);
            } else {
                const float W = ent[12];
                const float4 g = *reinterpret_cast<const float4*>(gsb + __float_as_int(ent[14]) * 32 + 4 * i - NRAW);
                v = make_float4(W * g.x, W * g.y, W * g.z, W * g.w);
            }
            red_add4(gacc + (size_t)k * GF + 4 * i, v);
        }
    }
}

// Fixed per-warp shared memory; the sample tables (RB * L entries) follow the
// array of these in dynamic shared memory.
struct alignas(16) WarpBwd {
    int4 task[TCAP];  // listed runs: (list entry, then primitive; ray slot / first / end sample; <gS, c>; 0)
    float queue[QCAP * QW];
    float gs[RB * 32];  // dL/dS of the bundle's rays, zero-padded
    int pre[32];        // inclusive prefix of list lengths over a chunk of samples
    int le[RB];         // composited samples of the bundle's rays
};

// Sample table of one warp, structure of arrays over RB * lmax samples.
struct Table {
    float4* xg;  // sample point, dL/dalpha_j
    int2* pv;    // packed voxel (ix | iy << 16, iz | start mask << 16); (0, -1) outside
    int2* nf;    // V_n, V_f of the voxel (0 outside)
    float* w;    // w_j = T_j alpha_j
};

// Run-start test of a sample's list entries against the previous sample's voxel:
// none start (same voxel, or no list), all start (first sample, or the previous
// one outside the grid), test each entry's range, or a mask of range-boundary
// flags (a step of at most two voxels per axis; entries start whose flags hit it).
constexpr int MK_NONE = 0, MK_ALL = 0x1000, MK_BOX = 0x2000, MK_FLAGS = 0xfff;

__device__ __forceinline__ int mask_of(int2 pv) { return pv.y < 0 ? MK_NONE : (int)((unsigned)pv.y >> 16); }

__host__ __device__ inline size_t table_stride(int lmax) { return ((size_t)RB * lmax * 36 + 15) / 16 * 16; }

__device__ __forceinline__ Table table_at(unsigned char* base, int lmax) {
    const size_t n = (size_t)RB * lmax;
    Table t;
    t.xg = reinterpret_cast<float4*>(base);
    t.pv = reinterpret_cast<int2*>(base + n * 16);
    t.nf = reinterpret_cast<int2*>(base + n * 24);
    t.w = reinterpret_cast<float*>(base + n * 32);
    return t;
}

// Start mask of a sample in voxel (ix, iy, iz) after one in voxel pv (packed).
__device__ __forceinline__ int start_mask(int2 cur, int2 prev, bool has_flags) {
    if (cur.y < 0) return MK_NONE;
    if (prev.y < 0) return MK_ALL;
    if (cur.x == prev.x && cur.y == prev.y) return MK_NONE;
    if (!has_flags) return MK_BOX;
    const int d[3] = {(cur.x & 0xffff) - (prev.x & 0xffff), (int)((unsigned)cur.x >> 16) - (int)((unsigned)prev.x >> 16),
                      cur.y - prev.y};
    int m = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 2 || d[a] < -2) return MK_BOX;
        const int bits = d[a] == 1 ? 1 : d[a] == 2 ? 3 : d[a] == -1 ? 4 : d[a] == -2 ? 12 : 0;
        m |= bits << (4 * a);
    }
    return m;
}

// Back-to-front sweep of every ray (one warp per ray, chunks of 32 samples):
// v_j = gD t_j + <gS, s_j> from the saved s_j, the carry
// U_j = alpha_{j+1} v_{j+1} + (1 - alpha_{j+1}) U_{j+1} as a 32-lane suffix scan of
// the affine maps U -> alpha v + (1 - alpha) U, then gw[r, j] = (dL/dalpha_j, w_j)
// with dL/dalpha_j = T_j (v_j - U_j) (0 where the clamp was active), w_j = T_j alpha_j.
template <int CP>
__global__ void __launch_bounds__(256) k_bwd_sweep(Batch B) {
    const int lane = threadIdx.x & 31;
    const long long nwarp = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long gr = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gr < B.total; gr += nwarp) {
        const int si = scene_of(B, gr);
        const SceneDesc& S = B.d[si];
        if (*S.status != SQ_OK || *S.save_status != SQ_OK) continue;
        const long long r = gr - __ldg(B.off + si);
        const int L = S.L, C = S.C;
        const int Le = min(max(__ldg(S.save_n + r), 0), L);
        const float gD = __ldg(S.grad_depth + r);
        const float gsl = lane < C ? __ldg(S.grad_sem + r * C + lane) : 0.f;
        float carry = 0.f;  // U at the last sample of the chunk being processed
        // the ray's page table: up to 32 entries held one per lane (read together
        // with the ray's counts), longer tables read per chunk
        const int* __restrict__ prow = S.save_page + r * S.save_np;
        const bool reg_table = S.save_np <= 32;
        const int pent = reg_table && lane < S.save_np ? __ldg(prow + lane) : -1;
        for (int jc = Le > 0 ? ((Le - 1) >> 5) << 5 : 0; Le > 0 && jc >= 0; jc -= 32) {
            const int j = jc + lane;
            const bool valid = j < Le;
            const int pidx = j / SAVE_PS;
            int pg = __shfl_sync(0xffffffffu, pent, pidx & 31);
            if (!reg_table) pg = valid ? __ldg(prow + pidx) : -1;
            if (valid && pg >= 0 && !SQ_BOUND(pg < S.save_cap, 3)) pg = -1;
            float sa = 0.f, T = 0.f, tj = 0.f;
            float4 sc[CP / 4];
#pragma unroll
            for (int q = 0; q < CP / 4; ++q) sc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid && pg >= 0) {
                const long long sj = (long long)pg * SAVE_PS + (j % SAVE_PS);
                const float2 ta = __ldg(S.save_TA + sj);
                T = ta.x;
                sa = ta.y;
                tj = __ldg(S.t + j);
                const float4* sv = S.save_S + sj * (CP / 4);
#pragma unroll
                for (int q = 0; q < CP / 4; ++q) sc[q] = __ldg(sv + q);
            }
            float dot = 0.f;  // <gS, s_j>; the padded classes of s_j are zero
#pragma unroll
            for (int q = 0; q < CP / 4; ++q) {
                dot = fmaf(__shfl_sync(0xffffffffu, gsl, 4 * q + 0), sc[q].x, dot);
                dot = fmaf(__shfl_sync(0xffffffffu, gsl, 4 * q + 1), sc[q].y, dot);
                dot = fmaf(__shfl_sync(0xffffffffu, gsl, 4 * q + 2), sc[q].z, dot);
                dot = fmaf(__shfl_sync(0xffffffffu, gsl, 4 * q + 3), sc[q].w, dot);
            }
            const float v = valid ? fmaf(gD, tj, dot) : 0.f;
            const float al = fabsf(sa);
            // f_j(U) = al v + (1 - al) U; after the scan (a, b) is f_j o ... o f_{jc+31}
            float a = al * v, b = 1.f - al;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const float a2 = __shfl_down_sync(0xffffffffu, a, o2);
                const float b2 = __shfl_down_sync(0xffffffffu, b, o2);
                if (lane + o2 < 32) {
                    a = fmaf(b, a2, a);
                    b *= b2;
                }
            }
            float na = __shfl_down_sync(0xffffffffu, a, 1), nb = __shfl_down_sync(0xffffffffu, b, 1);
            if (lane == 31) {
                na = 0.f;
                nb = 1.f;
            }
            const float U = fmaf(nb, carry, na);  // U_j
            if (valid) S.gw[r * L + j] = make_float2(sa < 0.f ? 0.f : T * (v - U), T * al);
            const float a0 = __shfl_sync(0xffffffffu, a, 0), b0 = __shfl_sync(0xffffffffu, b, 0);
            carry = fmaf(b0, carry, a0);
        }
    }
}

// Fills ray slot q of the table (one warp, chunks of 32 samples): sample point,
// voxel, its list, the run-start mask and the sweep's (dL/dalpha_j, w_j).
__device__ __forceinline__ void build_table(const SceneDesc& S, long long r, int q, int Le, const Table& tb,
                                            int lmax, int lane) {
    float o[3], d[3];
    scene_ray(S, r, o, d);
    const GridC g = S.g;
    const bool has_flags = S.v_flags != nullptr;
    const float2* __restrict__ gw = S.gw + r * S.L;
    int2 carry = make_int2(0, -1);  // voxel of the sample before the chunk (none yet)
    for (int jc = 0; jc < Le; jc += 32) {
        const int j = jc + lane;
        float x[3] = {0.f, 0.f, 0.f};
        int vi[3];
        int vox = -1;
        if (j < Le) vox = sample_voxel(g, o, d, __ldg(S.t + j), x, vi);
        const int2 pv = vox >= 0 ? make_int2(vi[0] | (vi[1] << 16), vi[2]) : make_int2(0, -1);
        int2 prev = make_int2(__shfl_up_sync(0xffffffffu, pv.x, 1), __shfl_up_sync(0xffffffffu, pv.y, 1));
        if (lane == 0) prev = carry;
        carry = make_int2(__shfl_sync(0xffffffffu, pv.x, 31), __shfl_sync(0xffffffffu, pv.y, 31));
        if (j < Le) {
            const float2 gwj = gw[j];
            int2 nf = make_int2(0, 0);
            if (vox >= 0) nf = make_int2(__ldg(S.v_n + vox), __ldg(S.v_f + vox));
            const int at = q * lmax + j;
            const int mk = nf.x > 0 ? start_mask(pv, prev, has_flags) : MK_NONE;
            tb.xg[at] = make_float4(x[0], x[1], x[2], gwj.x);
            tb.pv[at] = pv.y < 0 ? pv : make_int2(pv.x, pv.y | (mk << 16));
            tb.nf[at] = nf;
            tb.w[at] = gwj.y;
        }
    }
}

template <int CP>
__global__ void __launch_bounds__(MAX_WARPS * 32) k_backward(Batch B) {
    extern __shared__ __align__(16) unsigned char dyn[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int lmax = B.lmax;
    WarpBwd& sm = reinterpret_cast<WarpBwd*>(dyn)[wid];
    const Table tb = table_at(dyn + (size_t)nw * sizeof(WarpBwd) + (size_t)wid * table_stride(lmax), lmax);
    const long long nbund = __ldg(B.boff + B.n);

    for (;;) {
        int bb = 0;
        if (lane == 0) bb = atomicAdd(B.ctr, 1);
        const long long gb = __shfl_sync(0xffffffffu, bb, 0);
        if (gb >= nbund) break;
        int si = 0;
        {
            int lo = 0, hi = B.n;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(B.boff + mid) <= gb) lo = mid;
                else hi = mid;
            }
            si = lo;
        }
        const SceneDesc& S = B.d[si];
        if (*S.status != SQ_OK || *S.save_status != SQ_OK) continue;
        const long long r0 = (gb - __ldg(B.boff + si)) * RB;
        const int nr = (int)min((long long)RB, S.R - r0);
        const int C = S.C;
        __syncwarp();
        for (int q = 0; q < RB; ++q) {
            sm.gs[q * 32 + lane] = (q < nr && lane < C) ? __ldg(S.grad_sem + (r0 + q) * C + lane) : 0.f;
            if (lane == 0) sm.le[q] = q < nr ? min(max(__ldg(S.save_n + r0 + q), 0), S.L) : 0;
        }
        __syncwarp();
        for (int q = 0; q < nr; ++q) build_table(S, r0 + q, q, sm.le[q], tb, lmax, lane);
        __syncwarp();

        int qn = 0;                  // pending flushes
        int eq = 0, ec = 0, ee = 0;  // where the run listing resumes: ray slot, chunk, entry
        bool more = nr > 0;
        while (more) {
            // ---- list run starts until the task list is full or every run is listed:
            // the list entries of a chunk of 32 samples are numbered consecutively
            // and tested LU batches of 32 at a time
            int nt = 0;
            for (;;) {
                if (eq >= nr) {
                    more = false;
                    break;
                }
                const int Lq = sm.le[eq];
                if (ec * 32 >= Lq) {
                    ++eq;
                    ec = 0;
                    ee = 0;
                    continue;
                }
                const int j = ec * 32 + lane, at = eq * lmax + j;
                int nj = 0, fj = 0, mj = MK_NONE;
                if (j < Lq) {
                    mj = mask_of(tb.pv[at]);
                    if (mj != MK_NONE) {
                        const int2 nf = tb.nf[at];
                        nj = nf.x;
                        fj = nf.y;
                    }
                }
                const int incl = warp_incl_scan(nj, lane);
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                sm.pre[lane] = incl;
                __syncwarp();
                bool full = false;
                while (ee < tot && !full) {
                    int ent[LU], jl[LU], ml[LU];
                    unsigned fv[LU];
                    bool st[LU];
#pragma unroll
                    for (int u = 0; u < LU; ++u) {
                        const int e = ee + 32 * u + lane;
                        const bool valid = e < tot;
                        int l = 0;  // sample of entry e: number of prefixes <= e
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1)
                            if (sm.pre[l + step - 1] <= e) l += step;
                        // every lane takes part in both shuffles; invalid lanes drop the results
                        const int fl = __shfl_sync(0xffffffffu, fj, l);
                        const int ms = __shfl_sync(0xffffffffu, mj, l);
                        ml[u] = valid ? ms : MK_NONE;
                        jl[u] = ec * 32 + l;
                        ent[u] = valid ? fl + (e - (l > 0 ? sm.pre[l - 1] : 0)) : 0;
                        fv[u] = (ml[u] & MK_FLAGS) ? __ldg(S.v_flags + ent[u]) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < LU; ++u) {
                        st[u] = ml[u] == MK_ALL || (fv[u] & (unsigned)(ml[u] & MK_FLAGS)) != 0u;
                        if (ml[u] == MK_BOX) {
                            const int2 pl = tb.pv[eq * lmax + jl[u] - 1];
                            const int kk = __ldg(S.v_sq + ent[u]);
                            st[u] = SQ_BOUND((unsigned)kk < (unsigned)S.n, 2) ? !box_has(__ldg(S.boxes + kk), pl) : false;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < LU; ++u) {
                        if (nt + 32 > TCAP) {  // resume at batch u after the walk
                            full = true;
                            ee += 32 * u;
                            break;
                        }
                        const unsigned bm = __ballot_sync(0xffffffffu, st[u]);
                        if (st[u]) sm.task[nt + __popc(bm & lt)] = make_int4(ent[u], (eq << 16) | jl[u], 0, 0);
                        nt += __popc(bm);
                    }
                    if (!full) ee += 32 * LU;
                }
                __syncwarp();
                if (full) break;
                ++ec;
                ee = 0;
            }
            __syncwarp();
            // ---- per listed run, all lanes busy: its end (the samples in the
            // primitive's box form one interval, so a binary search finds the
            // last) and <gS, c_k> of its ray
            for (int t0 = 0; t0 < nt; t0 += 32 * RU) {
                // RU runs per lane, their loads in flight together
                int k[RU], q[RU], j0[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int t = t0 + 32 * u + lane;
                    k[u] = 0;
                    q[u] = 0;
                    j0[u] = 0;
                    if (t < nt) {
                        const int4 tk = sm.task[t];
                        q[u] = tk.y >> 16;
                        j0[u] = tk.y & 0xffff;
                        k[u] = __ldg(S.v_sq + tk.x);
                        if (!SQ_BOUND((unsigned)k[u] < (unsigned)S.n, 2)) k[u] = 0;
                    }
                }
                int4 box[RU];
                float cd[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    box[u] = __ldg(S.boxes + k[u]);
                    cd[u] = logit_dot<CP>(S.lpad, k[u], sm.gs + q[u] * 32);
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int t = t0 + 32 * u + lane;
                    if (t < nt) {
                        const int2* pv = tb.pv + q[u] * lmax;
                        int lo = j0[u], hi = sm.le[q[u]] - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (box_has(box[u], pv[mid])) lo = mid;
                            else hi = mid - 1;
                        }
                        sm.task[t] = make_int4(k[u], (q[u] << 21) | ((lo + 1) << 10) | j0[u], __float_as_int(cd[u]), 0);
                    }
                }
            }
            __syncwarp();
            // ---- walk the listed runs; idle lanes take the next runs together
            int next = 0;
            bool act = false;
            int k = 0, rq = 0, jj = 0, jend = 0;
            BwdPrim P;
            float cd = 0.f;
            float acc[13];
#pragma unroll
            for (int i = 0; i < 13; ++i) acc[i] = 0.f;
            for (;;) {
                const unsigned idle = __ballot_sync(0xffffffffu, !act);
                const int nidle = __popc(idle);
                if (next < nt && (nidle >= RTH || nidle == 32)) {
                    const int idx = next + __popc(idle & lt);
                    if (!act && idx < nt) {
                        const int4 tk = sm.task[idx];
                        k = tk.x;
                        rq = tk.y >> 21;
                        jend = (tk.y >> 10) & 2047;
                        jj = tk.y & 1023;
                        cd = __int_as_float(tk.z);
                        P = load_bwd(S.rec, S.aux, k);
#pragma unroll
                        for (int i = 0; i < 13; ++i) acc[i] = 0.f;
                        act = true;
                    }
                    next = min(next + nidle, nt);
                }
                if (!__any_sync(0xffffffffu, act)) break;
                bool ends = false;
                if (act) {
                    // NS samples of the run per step (independent chains)
                    const int at = rq * lmax + jj;
                    float po[NS], pr[NS][11];
                    float4 xg[NS];
                    float w[NS];
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        const bool in = jj + i < jend;
                        xg[i] = tb.xg[in ? at + i : at];
                        w[i] = in ? tb.w[at + i] : 0.f;
                        if (!in) xg[i].w = 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        const float x[3] = {xg[i].x, xg[i].y, xg[i].z};
                        po[i] = occupancy_partials(P, x, pr[i]);
                    }
#pragma unroll
                    for (int i = 0; i < NS; ++i)
                        if (jj + i < jend && po[i] != 0.f) accumulate(acc, po[i], pr[i], xg[i].w, w[i], P.f.sigma, cd);
                    jj = min(jj + NS, jend);
                    ends = jj >= jend;
                }
                const unsigned dm = __ballot_sync(0xffffffffu, ends);
                if (dm) {
                    if (qn + __popc(dm) > QCAP) {
                        __syncwarp();
                        drain_queue(S.gacc, sm.queue, qn, lane, sm.gs, C);
                        __syncwarp();
                        qn = 0;
                    }
                    if (ends) {
                        float4* ent = reinterpret_cast<float4*>(sm.queue + (qn + __popc(dm & lt)) * QW);
                        ent[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                        ent[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
                        ent[2] = make_float4(acc[8], acc[9], acc[10], acc[11]);
                        ent[3] = make_float4(acc[12], __int_as_float(k), __int_as_float(rq), 0.f);
                        act = false;
                    }
                    qn += __popc(dm);
                }
            }
            __syncwarp();
        }
        __syncwarp();
        drain_queue(S.gacc, sm.queue, qn, lane, sm.gs, C);
        __syncwarp();
    }
}

// Converts each primitive's summed partials into the six gradient outputs:
//   dL/dm = -sum gx;  dL/dq = (0, 2 tau) (x) qn / |q| (the torque of a world-frame
//   rotation mapped onto the tangent of the unit quaternion, then through q/|q|);
//   dL/ds_j = -sum(u_j df/du_j) / s_j;  dL/deps, dL/dsigma as summed;
//   dL/dc as accumulated.  One thread per primitive.
__global__ void k_grad_out(const float* __restrict__ gacc, const float4* __restrict__ aux,
                           const float* __restrict__ lpad, int cp, int sem_mode, int n, int C,
                           const int* __restrict__ status, const int* __restrict__ save_status,
                           float* __restrict__ gm, float* __restrict__ gq, float* __restrict__ gs,
                           float* __restrict__ ge, float* __restrict__ go, float* __restrict__ gl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (*status != SQ_OK || (save_status && *save_status != SQ_OK)) {
        // no work was done: zero gradients (the packed records may hold NaN)
        for (int i = 0; i < 3; ++i) gm[3 * k + i] = gs[3 * k + i] = 0.f;
        for (int i = 0; i < 4; ++i) gq[4 * k + i] = 0.f;
        ge[2 * k + 0] = ge[2 * k + 1] = go[k] = 0.f;
        for (int c = 0; c < C; ++c) gl[(size_t)k * C + c] = 0.f;
        return;
    }
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
    if (sem_mode == SQ_SEM_SOFTMAX) {
        // through s = softmax(c): dL/dc = s * (g - <g, s>), s as packed
        const float* sm = lpad + (size_t)k * cp;
        float gs_dot = 0.f;
        for (int c = 0; c < C; ++c) gs_dot = fmaf(e[NRAW + c], sm[c], gs_dot);
        for (int c = 0; c < C; ++c) gl[(size_t)k * C + c] = sm[c] * (e[NRAW + c] - gs_dot);
    } else {
        for (int c = 0; c < C; ++c) gl[(size_t)k * C + c] = e[NRAW + c];
    }
}


}  // namespace

int bwd_rays_per_bundle() { return RB; }

sq_status_t launch_sweep(const Batch& B, int cp, cudaStream_t st) {
    if (B.total == 0) return SQ_OK;
    const void* sw = nullptr;
    switch (cp) {
        case 4: sw = (const void*)k_bwd_sweep<4>; break;
        case 8: sw = (const void*)k_bwd_sweep<8>; break;
        case 12: sw = (const void*)k_bwd_sweep<12>; break;
        case 16: sw = (const void*)k_bwd_sweep<16>; break;
        case 20: sw = (const void*)k_bwd_sweep<20>; break;
        case 24: sw = (const void*)k_bwd_sweep<24>; break;
        case 28: sw = (const void*)k_bwd_sweep<28>; break;
        case 32: sw = (const void*)k_bwd_sweep<32>; break;
        default:
            set_last_error("n_classes padding %d not supported", cp);
            return SQ_ERR_INVALID_ARG;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sw, 256, 0);
    if (e != cudaSuccess) return cuda_status(e, "k_bwd_sweep occupancy");
    long long blocks = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    const long long need = (B.total + 7) / 8;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    Batch arg = B;
    void* args[] = {&arg};
    prof_begin("k_bwd_sweep", st);
    e = cudaLaunchKernel(sw, dim3((unsigned)blocks), dim3(256), args, 0, st);
    prof_end(st);
    if (e != cudaSuccess) return cuda_status(e, "k_bwd_sweep");
    return SQ_OK;
}

sq_status_t launch_backward(const Batch& B, int cp, const Tuning& tn, cudaStream_t st) {
    if (B.total == 0) return SQ_OK;
    int warps = tn.bwd_warps;  // 0: the count that keeps the most warps resident
    if (warps < 0 || warps > MAX_WARPS) {
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
    // per warp: fixed part plus a sample table of RB * lmax entries
    // shared memory per warp grows with the batch's largest L: the warps per CTA
    // decide how many CTAs fit on an SM
    const size_t per_warp = sizeof(WarpBwd) + table_stride(B.lmax);
    cudaError_t e;
    const size_t kMaxSmem = 227 * 1024;
    if (per_warp > kMaxSmem) {
        set_last_error("backward: %d samples per ray need %zu bytes of shared memory per warp", B.lmax, per_warp);
        return SQ_ERR_INVALID_ARG;
    }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return cuda_status(e, "k_backward shared memory");
    const int want = warps;
    int per_sm = 0, best_resident = -1;
    warps = 0;
    for (int w = MAX_WARPS; w >= 1; w >>= 1) {
        if ((want != 0 && w != want) || (size_t)w * per_warp > kMaxSmem) continue;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, w * 32, (size_t)w * per_warp);
        if (e != cudaSuccess) return cuda_status(e, "k_backward occupancy");
        if (b * w > best_resident) {
            best_resident = b * w;
            per_sm = b;
            warps = w;
        }
    }
    if (warps == 0) {  // the requested count does not fit: the largest power of two that does
        warps = 1;
        while (warps * 2 <= MAX_WARPS && (size_t)(warps * 2) * per_warp <= kMaxSmem) warps *= 2;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, (size_t)warps * per_warp);
        if (e != cudaSuccess) return cuda_status(e, "k_backward occupancy");
    }
    const size_t smem = (size_t)warps * per_warp;
    const long long need = (B.total / RB + B.n + warps - 1) / warps;
    long long blocks = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    Batch arg = B;
    void* args[] = {&arg};
    prof_begin("k_backward", st);
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(warps * 32), args, smem, st);
    prof_end(st);
    if (e != cudaSuccess) return cuda_status(e, "k_backward");
    return SQ_OK;
}

sq_status_t launch_grad_out(const SceneDesc& S, float* gm, float* gq, float* gs, float* ge, float* go, float* gl,
                            cudaStream_t st) {
    if (S.n == 0) return SQ_OK;
    SQ_LAUNCH("k_grad_out", st, k_grad_out<<<(S.n + 127) / 128, 128, 0, st>>>(S.gacc, S.aux, S.lpad, S.cp, S.sem_mode, S.n, S.C, S.status, S.save_status, gm, gq, gs, ge, go, gl));
    return SQ_OK;
}

sq_status_t launch_pack_boxes(const int* ranges, int n, int4* boxes, cudaStream_t st) {
    if (n == 0) return SQ_OK;
    SQ_LAUNCH("k_pack_boxes", st, k_pack_boxes<<<(n + 127) / 128, 128, 0, st>>>(ranges, n, boxes));
    return SQ_OK;
}

#ifdef SQR_CHECK
unsigned check_take_bwd() { return check_take(); }
#endif

}  // namespace sqr
