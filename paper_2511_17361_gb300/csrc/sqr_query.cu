// sqr_query.cu -- voxelisation of Supp. A.4 through the same index: at every
// voxel centre p, density = sum_{k in Q(v)} p_o(p, S_k) sigma_k and the semantic
// sum s = sum p_o c_k; label = argmax_c s (lowest index on ties) when density >= tau,
// otherwise "free" (= C).
//
// One lane per voxel; groups of Q_GROUP lanes (voxel ids are z-fastest, so the
// group's voxels are neighbours with near-identical lists) walk their lists
// together so that each record is loaded once per group.  The per-voxel semantic
// row is staged in shared memory so that the [nvox, C] output is written with
// coalesced stores.
//
// The backward (gradients of a loss on density and semantics) is primitive-major:
// primitive k is listed in exactly the voxels of its range, so a warp walks one
// of QB_SPLIT equal chunks of that range, sums dL/dp_o dp_o/dtheta over it in
// registers and adds its sums to the primitive's row once (one coalesced atomic
// add per chunk); k_grad_out converts the rows.
#include <limits.h>
#include <string.h>

#include "sqr_pair.cuh"
#include "sqr_render.cuh"

namespace sqr {

namespace {

constexpr int Q_THREADS = 128;
constexpr int Q_GROUP = 16;  // voxels (lanes) that walk their lists together (4 and 8 measured 2% slower)

struct QueryArgs {
    const float4* rec;
    const float* lpad;
    const int* v_n;
    const int* v_f;
    const int* v_sq;
    const int* status;
    GridC g;
    long long nvox;
    long long v_cap;  // entries V_sq holds
    int n;            // primitives
    int C;
    float tau;
    float* density;
    float* sem;
    unsigned char* label;
};

// Smallest id over a lane group of GQ lanes.
template <int GQ>
__device__ __forceinline__ int group_min(int k) {
#pragma unroll
    for (int o = GQ / 2; o > 0; o >>= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o, GQ));
    return k;
}

// A group of GQ lanes (GQ consecutive voxels, z-fastest: neighbours whose lists
// are nearly the same) walks the union of its sorted lists in ascending id: each
// step loads one record and class row for the whole group (the next step's record
// one step ahead) and the lanes whose list holds the id add its term.  Every voxel
// still sums its own list in ascending id order.
template <int CP, int GQ>
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
        float dens = 0.f, x[3] = {0.f, 0.f, 0.f};
        int n = 0, f = 0;
        if (v < a.nvox) {
            const int iz = (int)(v % nz);
            const int iy = (int)((v / nz) % ny);
            const int ix = (int)(v / ((long long)ny * nz));
            const int id[3] = {ix, iy, iz};
#pragma unroll
            for (int i = 0; i < 3; ++i)
                x[i] = __fadd_rn(a.g.lo[i], __fmul_rn(__fadd_rn(__int2float_rn(id[i]), 0.5f), a.g.vs[i]));
            n = __ldg(a.v_n + v);
            f = __ldg(a.v_f + v);
            if (n > 0 && !SQ_BOUND(f >= 0 && (long long)f + n <= a.v_cap, 1)) n = 0;
        }
        int e = 0;
        int head = n > 0 ? __ldg(a.v_sq + f) : INT_MAX;
        int head2 = n > 1 ? __ldg(a.v_sq + f + 1) : INT_MAX;
        int kmin = group_min<GQ>(head);
        Prim p;
        if (kmin != INT_MAX && SQ_BOUND((unsigned)kmin < (unsigned)a.n, 2)) p = load_prim(a.rec, kmin);
        while (__any_sync(0xffffffffu, kmin != INT_MAX)) {
            const int knext = group_min<GQ>(head == kmin ? head2 : head);
            Prim pn;
            if (knext != INT_MAX && SQ_BOUND((unsigned)knext < (unsigned)a.n, 2)) pn = load_prim(a.rec, knext);
            if (kmin != INT_MAX) {
                // (a listed id that is not a primitive is skipped, its list still advances)
                const bool idok = SQ_BOUND((unsigned)kmin < (unsigned)a.n, 2);
                const float4* cr = lp4 + (size_t)(idok ? kmin : 0) * (CP / 4);
                float4 cv[CP / 4];
#pragma unroll
                for (int q = 0; q < CP / 4; ++q) cv[q] = idok ? __ldg(cr + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (head == kmin) {
                    const float po = idok ? occupancy(p, x) : 0.f;
                    dens = fmaf(po, p.sigma, dens);
#pragma unroll
                    for (int q = 0; q < CP / 4; ++q) {
                        acc[4 * q + 0] = fmaf(po, cv[q].x, acc[4 * q + 0]);
                        acc[4 * q + 1] = fmaf(po, cv[q].y, acc[4 * q + 1]);
                        acc[4 * q + 2] = fmaf(po, cv[q].z, acc[4 * q + 2]);
                        acc[4 * q + 3] = fmaf(po, cv[q].w, acc[4 * q + 3]);
                    }
                    ++e;
                    head = head2;
                    head2 = e + 1 < n ? __ldg(a.v_sq + f + e + 1) : INT_MAX;
                }
            }
            kmin = knext;
            p = pn;
        }
        if (v < a.nvox) {
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
        for (long long e2 = threadIdx.x; e2 < total; e2 += Q_THREADS) {
            const int row = (int)(e2 / a.C), c = (int)(e2 - (long long)row * a.C);
            out[e2] = rows[row * (CP + 1) + c];
        }
        __syncthreads();
    }
}

// Tile-major form of the same sums.  A block takes a tile of QT_X x QT_Y x QT_Z
// voxels, one voxel per thread.  It scans the primitives' packed voxel ranges in
// rounds of QT_ROUND ids, warp w the w-th window of QT_WIN ids of the round,
// and keeps those that meet the tile, each with the tile-local bit masks of its
// x, y and z extent; the warps' lists, in warp order, are the round's list in id
// order.  Then, QT_STAGE primitives at a time, it stages their records and class
// rows in shared memory.  Every thread
// adds the terms of the primitives whose range holds its voxel.  A voxel's
// list Q(v) is exactly the primitives whose range holds v, so every voxel still
// sums its own list in ascending id order: the sums are those of k_query.
// Warp w holds a 4 x 4 x 2 block of the tile: compact blocks leave fewer lanes
// idle where a range covers part of a warp (about 19% of the lanes of evaluating
// warps on the 8192-superquadric scene, against 25% for 8 x 4 x 1 rows).
constexpr int QT_X = 8, QT_Y = 8, QT_Z = 4;
constexpr int QT_THREADS = QT_X * QT_Y * QT_Z;
constexpr int QT_WIN = 128;                           // ids a warp scans per round
constexpr int QT_ROUND = QT_WIN * (QT_THREADS / 32);  // ids per round
constexpr int QT_STAGE = 64;                          // primitives staged in shared memory at a time
static_assert(QT_THREADS == 256 && QT_WIN % 32 == 0, "tile shape");
static_assert(QT_X == 8 && QT_Y == 8 && QT_Z == 4, "warps of 4 x 4 x 2 voxels; 8-bit extent masks");

template <int CP>
struct QtSmem {
    int wid_[QT_THREADS / 32][QT_WIN];       // each warp's hits of the round, in id order
    unsigned wmsk[QT_THREADS / 32][QT_WIN];  // x extent bits 0-7, y bits 8-15, z bits 16-23 (tile-local)
    int id[QT_ROUND];                         // the round's hits in id order
    unsigned msk[QT_ROUND];
    union {
        struct {
            float4 rec[QT_STAGE][REC4];
            float4 cls[QT_STAGE][CP / 4];
        } st;
        float rows[QT_THREADS * (CP + 1)];  // the tile's semantic rows, for coalesced stores
    } u;
    int wtot[QT_THREADS / 32];
};

// Bits lo..hi of a tile-local extent (empty when hi < lo).
__device__ __forceinline__ unsigned span_bits(int lo, int hi) {
    return hi < lo ? 0u : (2u << hi) - (1u << lo);
}

template <int CP>
__global__ void __launch_bounds__(QT_THREADS) k_query_tiles(QueryArgs a, const int4* __restrict__ boxes, int n,
                                                            int ntx, int nty, int ntz) {
    __shared__ QtSmem<CP> sh;
    if (*a.status != SQ_OK) return;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int lx = (wid & 1) * 4 + (lane & 3), ly = ((wid >> 1) & 1) * 4 + ((lane >> 2) & 3),
              lz = (wid >> 2) * 2 + (lane >> 4);
    const int lv = (lz * QT_Y + ly) * QT_X + lx;  // the voxel's row in the tile's staged rows
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const float4* lp4 = reinterpret_cast<const float4*>(a.lpad);
    for (int tile = blockIdx.x; tile < ntx * nty * ntz; tile += gridDim.x) {
        const int tz = tile % ntz, ty = (tile / ntz) % nty, tx = tile / (ntz * nty);
        const int x0 = tx * QT_X, y0 = ty * QT_Y, z0 = tz * QT_Z;
        const int x1 = min(x0 + QT_X, nx) - 1, y1 = min(y0 + QT_Y, ny) - 1, z1 = min(z0 + QT_Z, nz) - 1;
        const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
        const bool valid = ix <= x1 && iy <= y1 && iz <= z1;
        float x[3];
        {
            const int id3[3] = {ix, iy, iz};
#pragma unroll
            for (int i = 0; i < 3; ++i)
                x[i] = __fadd_rn(a.g.lo[i], __fmul_rn(__fadd_rn(__int2float_rn(id3[i]), 0.5f), a.g.vs[i]));
        }
        float acc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = 0.f;
        float dens = 0.f;
        const unsigned sel = (1u << lx) | (1u << (8 + ly)) | (1u << (16 + lz));  // this voxel's bits
        for (int r0 = 0; r0 < n; r0 += QT_ROUND) {
            // ---- warp wid: the primitives of its window that meet the tile, in id order
            int wc = 0;
#pragma unroll
            for (int s2 = 0; s2 < QT_WIN / 32; ++s2) {
                const int k = r0 + wid * QT_WIN + s2 * 32 + lane;
                unsigned m = 0u;
                if (k < n) {
                    const int4 b = __ldg(boxes + k);
                    const int bx0 = b.x & 0xffff, bx1 = (int)((unsigned)b.x >> 16);
                    const int by0 = b.y & 0xffff, by1 = (int)((unsigned)b.y >> 16);
                    const int bz0 = b.z & 0xffff, bz1 = (int)((unsigned)b.z >> 16);
                    if (bx0 <= x1 && bx1 >= x0 && by0 <= y1 && by1 >= y0 && bz0 <= z1 && bz1 >= z0 &&
                        bx0 <= bx1 && by0 <= by1 && bz0 <= bz1)
                        m = span_bits(max(bx0, x0) - x0, min(bx1, x1) - x0) |
                            (span_bits(max(by0, y0) - y0, min(by1, y1) - y0) << 8) |
                            (span_bits(max(bz0, z0) - z0, min(bz1, z1) - z0) << 16);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, m != 0u);
                if (m != 0u) {
                    const int pos = wc + __popc(bal & ((1u << lane) - 1u));
                    sh.wid_[wid][pos] = k;
                    sh.wmsk[wid][pos] = m;
                }
                wc += __popc(bal);
            }
            if (lane == 0) sh.wtot[wid] = wc;
            __syncthreads();
            // ---- the round's list: the warps' lists in warp order
            int before = 0, nc = 0;
#pragma unroll
            for (int w2 = 0; w2 < QT_THREADS / 32; ++w2) {
                const int v = sh.wtot[w2];
                before += w2 < wid ? v : 0;
                nc += v;
            }
            for (int j = lane; j < wc; j += 32) {
                sh.id[before + j] = sh.wid_[wid][j];
                sh.msk[before + j] = sh.wmsk[wid][j];
            }
            __syncthreads();
            // ---- the listed primitives' terms, QT_STAGE at a time
            for (int j0 = 0; j0 < nc; j0 += QT_STAGE) {
                const int nj = min(QT_STAGE, nc - j0);
                constexpr int PER = REC4 + CP / 4;
                for (int i = t; i < nj * PER; i += QT_THREADS) {
                    const int j = i / PER, q = i - j * PER;
                    const int kk = sh.id[j0 + j];
                    if (q < REC4) sh.u.st.rec[j][q] = __ldg(a.rec + (size_t)kk * REC4 + q);
                    else sh.u.st.cls[j][q - REC4] = __ldg(lp4 + (size_t)kk * (CP / 4) + (q - REC4));
                }
                __syncthreads();
                for (int j = 0; j < nj; ++j) {
                    // the warp evaluates when any of its voxels is in the range; the
                    // others add an exact zero (p_o is finite at every point)
                    const bool mem = (sh.msk[j0 + j] & sel) == sel;
                    if (__any_sync(0xffffffffu, mem)) {
                        const float4 r0v = sh.u.st.rec[j][0], r1 = sh.u.st.rec[j][1], r2 = sh.u.st.rec[j][2],
                                     r3 = sh.u.st.rec[j][3];
                        Prim p;
                        p.m[0] = r0v.x; p.m[1] = r0v.y; p.m[2] = r0v.z; p.sigma = r0v.w;
                        p.M[0][0] = r1.x; p.M[0][1] = r1.y; p.M[0][2] = r1.z; p.ea = r1.w;
                        p.M[1][0] = r2.x; p.M[1][1] = r2.y; p.M[1][2] = r2.z; p.eb = r2.w;
                        p.M[2][0] = r3.x; p.M[2][1] = r3.y; p.M[2][2] = r3.z; p.ec = r3.w;
                        const float pv = occupancy(p, x);
                        const float po = mem ? pv : 0.f;
                        dens = fmaf(po, p.sigma, dens);
#pragma unroll
                        for (int q = 0; q < CP / 4; ++q) {
                            const float4 cv = sh.u.st.cls[j][q];
                            acc[4 * q + 0] = fmaf(po, cv.x, acc[4 * q + 0]);
                            acc[4 * q + 1] = fmaf(po, cv.y, acc[4 * q + 1]);
                            acc[4 * q + 2] = fmaf(po, cv.z, acc[4 * q + 2]);
                            acc[4 * q + 3] = fmaf(po, cv.w, acc[4 * q + 3]);
                        }
                    }
                }
                __syncthreads();
            }
        }
        // ---- outputs: density and label per thread; the semantic rows through shared
        // memory, one warp per column (x, y) of the tile, whose z voxels' rows are
        // contiguous in [nvox, C]
        if (valid) {
            const long long v = ((long long)ix * ny + iy) * nz + iz;
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
        for (int c = 0; c < CP; ++c) sh.u.rows[lv * (CP + 1) + c] = acc[c];
        __syncthreads();
        {
            const int ncy = y1 - y0 + 1, ncol = (x1 - x0 + 1) * ncy, nzt = z1 - z0 + 1;
            for (int col = wid; col < ncol; col += QT_THREADS / 32) {
                const int cx = col / ncy, cy = col - cx * ncy;
                float* out = a.sem + (((long long)(x0 + cx) * ny + (y0 + cy)) * nz + z0) * a.C;
                for (int vz = 0; vz < nzt; ++vz) {
                    const float* row = sh.u.rows + (vz * (QT_X * QT_Y) + cy * QT_X + cx) * (CP + 1);
                    for (int c = lane; c < a.C; c += 32) out[vz * a.C + c] = row[c];
                }
            }
        }
        __syncthreads();
    }
}

constexpr int QB_THREADS = 256;
constexpr int QB_SPLIT = 8;  // chunks per primitive range (ranges differ widely in size)

struct QueryBwdArgs {
    const float4* rec;
    const float4* aux;
    const float* lpad;
    const int* ranges;
    const int* status;
    GridC g;
    int n, C;
    const float* grad_density;
    const float4* gsp;  // [nvox, CP/4] grad_sem rows zero-padded to CP classes
    float* gacc;  // [n, GF] raw sums, zeroed
    int* ctr;     // zeroed work counter over (primitive, chunk)
};

// grad_sem [V, C] copied to rows of CP classes (zero padding), one thread per
// (voxel, group of four classes): threadIdx.x the group, threadIdx.y the voxel,
// so that a pair reads its voxel's row with CP / 4 vector loads.
__global__ void k_pad_rows(const float* __restrict__ in, long long rows, int C, int cp4, float4* __restrict__ out) {
    const long long r = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (r >= rows) return;
    const int q = (int)threadIdx.x;
    const long long i = r * cp4 + q;
    float v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = 4 * q + c < C ? __ldg(in + r * C + 4 * q + c) : 0.f;
    out[i] = make_float4(v[0], v[1], v[2], v[3]);
}

// One warp per (primitive, chunk of its range), drawn from a counter: over the
// voxels v of the chunk, dL/dp_o = gd[v] sigma + <gs[v], c>; the row gets the 11
// summed partials of f weighted by -p_o dL/dp_o, sum gd p_o (opacity) and
// sum p_o gs[v, c] (logits).
template <int CP>
__global__ void __launch_bounds__(QB_THREADS) k_query_bwd(QueryBwdArgs a) {
    const int lane = threadIdx.x & 31;
    const bool ok = *a.status == SQ_OK;
    const int ny = a.g.n[1], nz = a.g.n[2];
    for (;;) {
        int ww = 0;
        if (lane == 0) ww = atomicAdd(a.ctr, 1);
        const int w = __shfl_sync(0xffffffffu, ww, 0);
        if (w >= a.n * QB_SPLIT) break;
        const int k = w / QB_SPLIT, part = w - k * QB_SPLIT;
        const int* r = a.ranges + 6 * k;
        const int i0 = __ldg(r), i1 = __ldg(r + 1), j0 = __ldg(r + 2), j1 = __ldg(r + 3), k0 = __ldg(r + 4),
                  k1 = __ldg(r + 5);
        const int nxb = i1 - i0 + 1, nyb = j1 - j0 + 1, nzb = k1 - k0 + 1;
        const long long nvb = (ok && nxb > 0 && nyb > 0 && nzb > 0) ? (long long)nxb * nyb * nzb : 0;
        const long long t_beg = nvb * part / QB_SPLIT, t_end = nvb * (part + 1) / QB_SPLIT;
        if (t_beg >= t_end) continue;
        float acc[NRAW];
        float accl[CP];
#pragma unroll
        for (int i = 0; i < NRAW; ++i) acc[i] = 0.f;
#pragma unroll
        for (int c = 0; c < CP; ++c) accl[c] = 0.f;
        {
            const BwdPrim P = load_bwd(a.rec, a.aux, k);
            float cl[CP];
            const float4* cr = reinterpret_cast<const float4*>(a.lpad) + (size_t)k * (CP / 4);
#pragma unroll
            for (int q = 0; q < CP / 4; ++q) {
                const float4 c4 = __ldg(cr + q);
                cl[4 * q] = c4.x;
                cl[4 * q + 1] = c4.y;
                cl[4 * q + 2] = c4.z;
                cl[4 * q + 3] = c4.w;
            }
            // the lane's voxel (ix, iy, iz) of range offset t, advanced by 32 offsets per
            // step as a mixed-radix sum (z fastest): no division inside the loop
            const long long t_first = t_beg + lane;
            int oz = (int)(t_first % nzb);
            const long long rest0 = t_first / nzb;
            int oy = (int)(rest0 % nyb), ox = (int)(rest0 / nyb);
            const int dz = 32 % nzb, dyz = 32 / nzb, dy = dyz % nyb, dx = dyz / nyb;
            for (long long t = t_first; t < t_end; t += 32) {
                const int iz = k0 + oz, iy = j0 + oy, ix = i0 + ox;
                oz += dz;
                const int cy = oz >= nzb ? 1 : 0;
                oz -= cy * nzb;
                oy += dy + cy;
                const int cx = oy >= nyb ? 1 : 0;
                oy -= cx * nyb;
                ox += dx + cx;
                const long long v = ((long long)ix * ny + iy) * nz + iz;
                const int id[3] = {ix, iy, iz};
                float x[3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    x[i] = __fadd_rn(a.g.lo[i], __fmul_rn(__fadd_rn(__int2float_rn(id[i]), 0.5f), a.g.vs[i]));
                const float gd = __ldg(a.grad_density + v);
                float gs[CP];
                float cd = 0.f;
                const float4* gr = a.gsp + v * (CP / 4);
#pragma unroll
                for (int q = 0; q < CP / 4; ++q) {
                    const float4 g4 = __ldg(gr + q);
                    gs[4 * q] = g4.x;
                    gs[4 * q + 1] = g4.y;
                    gs[4 * q + 2] = g4.z;
                    gs[4 * q + 3] = g4.w;
                }
#pragma unroll
                for (int c = 0; c < CP; ++c) cd = fmaf(gs[c], cl[c], cd);
                float pr[11];
                const float po = occupancy_partials(P, x, pr);
                if (po != 0.f) {
                    const float gf = -po * fmaf(gd, P.f.sigma, cd);
#pragma unroll
                    for (int i = 0; i < 11; ++i) acc[i] = fmaf(gf, pr[i], acc[i]);
                    acc[11] = fmaf(gd, po, acc[11]);
#pragma unroll
                    for (int c = 0; c < CP; ++c) accl[c] = fmaf(po, gs[c], accl[c]);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int i = 0; i < NRAW; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
#pragma unroll
            for (int c = 0; c < CP; ++c) accl[c] += __shfl_xor_sync(0xffffffffu, accl[c], o);
        }
        float* row = a.gacc + (size_t)k * GF;
        float v0 = 0.f, v1 = 0.f;  // lane f adds field f and f + 32
#pragma unroll
        for (int i = 0; i < NRAW; ++i)
            if (lane == i) v0 = acc[i];
#pragma unroll
        for (int c = 0; c < CP; ++c) {
            if (lane == NRAW + c) v0 = accl[c];
            if (lane + 32 == NRAW + c) v1 = accl[c];
        }
        if (lane < NRAW + a.C && v0 != 0.f) red_add(row + lane, v0);
        if (lane + 32 < NRAW + a.C && v1 != 0.f) red_add(row + 32 + lane, v1);
    }
}

}  // namespace

size_t render_workspace_size(const sq_prims_t* p);

// The grid query's workspace: the render workspace's per-primitive blocks (records,
// padded logits, accumulator, a counter: the backward's layout stays inside it),
// then for the backward the cotangent rows of every voxel padded to CP classes.
size_t query_workspace_size(const sq_prims_t* p, const sq_grid_t* g) {
    const long long nvox = (long long)g->nx * g->ny * g->nz;
    return align_up(render_workspace_size(p), 256) + align_up((size_t)nvox * cpad(p->n_classes) * sizeof(float), 256);
}

template <int CP>
static sq_status_t launch_query_cp(const QueryArgs& a, const int4* boxes, int n, cudaStream_t st) {
    if (boxes) {  // tile-major
        const int ntx = (a.g.n[0] + QT_X - 1) / QT_X, nty = (a.g.n[1] + QT_Y - 1) / QT_Y,
                  ntz = (a.g.n[2] + QT_Z - 1) / QT_Z;
        const long long ntiles = (long long)ntx * nty * ntz;
        const int blocks = (int)(ntiles < (1LL << 30) ? ntiles : (1LL << 30));
        SQ_LAUNCH("k_query_tiles", st, k_query_tiles<CP><<<blocks, QT_THREADS, 0, st>>>(a, boxes, n, ntx, nty, ntz));
        return SQ_OK;
    }
    long long want = (a.nvox + Q_THREADS - 1) / Q_THREADS;
    int blocks = (int)(want < 152LL * 64 ? want : 152LL * 64);
    if (blocks < 1) blocks = 1;
    SQ_LAUNCH("k_query", st, k_query<CP, Q_GROUP><<<blocks, Q_THREADS, 0, st>>>(a));
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
    // packed records at the start of the workspace, padded logits after them, then
    // the packed voxel ranges (inside the render workspace's per-primitive blocks)
    char* base = (char*)ws;
    float4* rec = (float4*)base;
    const size_t lp_at = align_up((size_t)prims->n * REC4 * sizeof(float4), 256);
    float* lpad = (float*)(base + lp_at);
    const size_t bx_at = lp_at + align_up((size_t)prims->n * cp * sizeof(float), 256);
    int4* boxes = nullptr;
    if (grid->nx <= 65535 && grid->ny <= 65535 && grid->nz <= 65535 && prims->n > 0 &&
        bx_at + (size_t)prims->n * sizeof(int4) <= need) {
        boxes = (int4*)(base + bx_at);
        sq_status_t sb = launch_pack_boxes(idx->ranges, prims->n, boxes, st);
        if (sb != SQ_OK) return sb;
    }
    sq_status_t s = launch_pack(prims, rec, nullptr, lpad, cp, st);
    if (s != SQ_OK) return s;
    QueryArgs a;
    a.rec = rec;
    a.lpad = lpad;
    a.v_n = idx->v_n;
    a.v_f = idx->v_f;
    a.v_sq = idx->v_sq;
    a.v_cap = idx->capacity;
    a.n = prims->n;
    a.status = idx->status;
    a.g = make_grid(grid);
    a.nvox = (long long)grid->nx * grid->ny * grid->nz;
    a.C = prims->n_classes;
    a.tau = tau;
    a.density = density;
    a.sem = sem;
    a.label = label;
    switch (cp) {
        case 4: return launch_query_cp<4>(a, boxes, prims->n, st);
        case 8: return launch_query_cp<8>(a, boxes, prims->n, st);
        case 12: return launch_query_cp<12>(a, boxes, prims->n, st);
        case 16: return launch_query_cp<16>(a, boxes, prims->n, st);
        case 20: return launch_query_cp<20>(a, boxes, prims->n, st);
        case 24: return launch_query_cp<24>(a, boxes, prims->n, st);
        case 28: return launch_query_cp<28>(a, boxes, prims->n, st);
        case 32: return launch_query_cp<32>(a, boxes, prims->n, st);
        default: return SQ_ERR_INVALID_ARG;
    }
}

template <int CP>
static sq_status_t launch_query_bwd_cp(const QueryBwdArgs& a, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_query_bwd<CP>, QB_THREADS, 0);
    if (e != cudaSuccess) return cuda_status(e, "k_query_bwd occupancy");
    long long blocks = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    const long long need = ((long long)a.n * QB_SPLIT + QB_THREADS / 32 - 1) / (QB_THREADS / 32);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    SQ_LAUNCH("k_query_bwd", st, k_query_bwd<CP><<<(int)blocks, QB_THREADS, 0, st>>>(a));
    return SQ_OK;
}

// Workspace of the query backward: records, backward extras, padded logits, the
// accumulator rows and a counter (within render_workspace_size).
sq_status_t query_grid_bwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                                const float* grad_density, const float* grad_sem, float* g_means, float* g_quats,
                                float* g_scales, float* g_eps, float* g_opacity, float* g_logits, void* ws,
                                size_t ws_bytes, cudaStream_t st) {
    const size_t need = query_workspace_size(prims, grid);
    if (ws == nullptr || ws_bytes < need) {
        set_last_error("sq_query_grid_bwd: workspace of %zu bytes given, %zu needed", ws_bytes, need);
        return SQ_ERR_INVALID_ARG;
    }
    const int n = prims->n, cp = cpad(prims->n_classes);
    if (n == 0) return SQ_OK;
    char* base = (char*)ws;
    size_t at = 0;
    float4* rec = (float4*)(base + at);
    at = align_up(at + (size_t)n * REC4 * sizeof(float4), 256);
    float4* aux = (float4*)(base + at);
    at = align_up(at + (size_t)n * AUX4 * sizeof(float4), 256);
    float* lpad = (float*)(base + at);
    at = align_up(at + (size_t)n * cp * sizeof(float), 256);
    float* gacc = (float*)(base + at);
    at = align_up(at + (size_t)n * GF * sizeof(float), 256);
    int* ctr = (int*)(base + at);
    at = align_up(at + sizeof(int), 256);
    float4* gsp = (float4*)(base + at);  // after the render workspace's blocks (query_workspace_size)
    const long long nvox = (long long)grid->nx * grid->ny * grid->nz;
    sq_status_t s = launch_pack(prims, rec, aux, lpad, cp, st);
    if (s != SQ_OK) return s;
    SQ_LAUNCH("k_pad_rows", st,
              k_pad_rows<<<(unsigned)((nvox + 63) / 64), dim3(cp / 4, 64), 0, st>>>(grad_sem, nvox, prims->n_classes,
                                                                                   cp / 4, gsp));
    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e, "memset counter");
    e = cudaMemsetAsync(gacc, 0, (size_t)n * GF * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "memset accumulator");
    QueryBwdArgs a;
    a.rec = rec;
    a.aux = aux;
    a.lpad = lpad;
    a.ranges = idx->ranges;
    a.status = idx->status;
    a.g = make_grid(grid);
    a.n = n;
    a.C = prims->n_classes;
    a.grad_density = grad_density;
    a.gsp = gsp;
    a.gacc = gacc;
    a.ctr = ctr;
    switch (cp) {
        case 4: s = launch_query_bwd_cp<4>(a, st); break;
        case 8: s = launch_query_bwd_cp<8>(a, st); break;
        case 12: s = launch_query_bwd_cp<12>(a, st); break;
        case 16: s = launch_query_bwd_cp<16>(a, st); break;
        case 20: s = launch_query_bwd_cp<20>(a, st); break;
        case 24: s = launch_query_bwd_cp<24>(a, st); break;
        case 28: s = launch_query_bwd_cp<28>(a, st); break;
        case 32: s = launch_query_bwd_cp<32>(a, st); break;
        default: return SQ_ERR_INVALID_ARG;
    }
    if (s != SQ_OK) return s;
    SceneDesc S;
    memset(&S, 0, sizeof(S));
    S.gacc = gacc;
    S.aux = aux;
    S.lpad = lpad;
    S.cp = cp;
    S.sem_mode = prims->sem_mode;
    S.n = n;
    S.C = prims->n_classes;
    S.status = idx->status;
    return launch_grad_out(S, g_means, g_quats, g_scales, g_eps, g_opacity, g_logits, st);
}

#ifdef SQR_CHECK
unsigned check_take_query() { return check_take(); }
#endif

}  // namespace sqr
