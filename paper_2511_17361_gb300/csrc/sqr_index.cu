// sqr_index.cu -- the voxel -> superquadric index of Sec. 3.3.1 ("Preliminary
// Construction"): V_n (count per voxel), V_f (offset per voxel) and V_sq
// (primitive ids per voxel, ascending), built on the GPU without any host sync.
//
//   1. k_ranges     one thread per primitive: the check of its parameters' domain
//                   (SQ_ERR_NUMERIC in the status word), its inclusive voxel box, in
//                   FP64 with explicitly rounded operations (bit-reproducible), and
//                   the 8 signed corner updates of a 3-D difference array;
//   2. k_prefix_*   three axis-wise prefix sums turn the difference array into V_n;
//   3. k_scan_*     exclusive scan of V_n -> V_f and the total P (+ capacity check);
//   4. k_scatter    one CTA per primitive writes its id into every voxel of its box
//                   at V_f[v] + (atomic cursor);
//   5. k_sort       one warp per voxel sorts its list ascending (bitonic network in
//                   registers, shared memory, or global memory by list length).
#include <math.h>
#include <stdio.h>

#include "sqr_common.cuh"
#include "sqr_render.cuh"

namespace sqr {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SORT_WARPS = 8;
constexpr int SORT_SMEM = 1024;  // per-warp list capacity staged in shared memory

struct RangeArgs {
    const float* means;
    const float* quats;
    const float* scales;
    const float* eps;
    const float* opacity;
    const float* logits;
    int C;
    int* status;
    int n;
    int mode;
    int nv;
    double log_kc;   // ln(ln(1/tau_cut)), computed on the host
    double tau;      // tau_cut (opacity-aware mode)
    double log_tau;  // ln(tau_cut), computed on the host
    int gn[3];
    double glo[3];
    double gvs[3];
};

// Voxel box of one primitive.  OBB mode: the level set p_o >= tau_cut lies in the
// local box |x_i| <= s_i Kc^(eps1/2) (Kc = ln(1/tau_cut)); its world AABB has
// half-width sum_i |R_ji| h_i.  Cube mode: centre voxel +- nv.  Clipped to the grid.
__device__ void prim_box(const RangeArgs& a, int k, int lo_i[3], int hi_i[3], bool& empty) {
    double w = a.quats[4 * k + 0], x = a.quats[4 * k + 1], y = a.quats[4 * k + 2], z = a.quats[4 * k + 3];
    double nq = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(w, w), __dmul_rn(x, x)), __dmul_rn(y, y)),
                                     __dmul_rn(z, z)));
    w = __ddiv_rn(w, nq);
    x = __ddiv_rn(x, nq);
    y = __ddiv_rn(y, nq);
    z = __ddiv_rn(z, nq);
    double R[9];
    R[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, y), __dmul_rn(z, z))));
    R[1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
    R[2] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
    R[3] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
    R[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(z, z))));
    R[5] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
    R[6] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
    R[7] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
    R[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))));
    double e1 = a.eps[2 * k + 0];
    double log_kc = a.log_kc;
    if (a.mode == SQ_INDEX_OBB_OPACITY) {
        // the level set sigma p_o >= tau_cut: Kc = ln(sigma) - ln(tau_cut); none if sigma <= tau_cut
        const double sig = a.opacity[k];
        if (!(sig > a.tau)) {
            empty = true;
            for (int j = 0; j < 3; ++j) {
                lo_i[j] = 0;
                hi_i[j] = -1;
            }
            return;
        }
        log_kc = log(__dsub_rn(log(sig), a.log_tau));
    }
    double ext = exp(__dmul_rn(__dmul_rn(0.5, e1), log_kc));
    double h[3];
    for (int i = 0; i < 3; ++i) h[i] = __dmul_rn((double)a.scales[3 * k + i], ext);
    empty = false;
    for (int j = 0; j < 3; ++j) {
        double m = a.means[3 * k + j];
        double ulo, uhi;
        if (a.mode != SQ_INDEX_CUBE) {
            double hw = __dadd_rn(__dmul_rn(fabs(R[3 * j + 0]), h[0]), __dmul_rn(fabs(R[3 * j + 1]), h[1]));
            hw = __dadd_rn(hw, __dmul_rn(fabs(R[3 * j + 2]), h[2]));
            ulo = __ddiv_rn(__dsub_rn(__dsub_rn(m, hw), a.glo[j]), a.gvs[j]);
            uhi = __ddiv_rn(__dsub_rn(__dadd_rn(m, hw), a.glo[j]), a.gvs[j]);
        } else {
            double uc = __ddiv_rn(__dsub_rn(m, a.glo[j]), a.gvs[j]);
            double cf = floor(fmin(fmax(uc, -1.0 - a.nv), (double)a.gn[j] + a.nv));
            ulo = cf - a.nv;
            uhi = cf + a.nv;
        }
        if (isnan(ulo) || isnan(uhi)) {
            empty = true;
            lo_i[j] = 0;
            hi_i[j] = -1;
            continue;
        }
        int i0 = (int)floor(fmin(fmax(ulo, -1.0), (double)a.gn[j]));
        int i1 = (int)floor(fmin(fmax(uhi, -1.0), (double)a.gn[j]));
        i0 = max(i0, 0);
        i1 = min(i1, a.gn[j] - 1);
        if (i0 > i1) empty = true;
        lo_i[j] = i0;
        hi_i[j] = i1;
    }
}

// The parameter domain of one superquadric (sq_prims_t): every value finite, a
// quaternion of non-zero length, scales > 0, eps1 and eps2 in (0, 2].
__device__ bool params_in_domain(const RangeArgs& a, int k) {
    bool ok = true;
    float q2 = 0.f;
    for (int i = 0; i < 3; ++i) {
        const float m = a.means[3 * k + i], s = a.scales[3 * k + i];
        ok = ok && isfinite(m) && isfinite(s) && s > 0.f;
    }
    for (int i = 0; i < 4; ++i) {
        const float q = a.quats[4 * k + i];
        ok = ok && isfinite(q);
        q2 = fmaxf(q2, fabsf(q));
    }
    for (int i = 0; i < 2; ++i) {
        const float e = a.eps[2 * k + i];
        ok = ok && e > 0.f && e <= 2.f;  // false for NaN
    }
    ok = ok && q2 > 0.f && isfinite(a.opacity[k]);
    for (int c = 0; c < a.C; ++c) ok = ok && isfinite(a.logits[(size_t)k * a.C + c]);
    return ok;
}

__global__ void k_ranges(RangeArgs a, int* __restrict__ ranges, int* __restrict__ diff) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    if (!params_in_domain(a, k)) atomicMax(a.status, (int)SQ_ERR_NUMERIC);
    int lo[3], hi[3];
    bool empty;
    prim_box(a, k, lo, hi, empty);
    int* r = ranges + 6 * k;
    if (empty) {
        r[0] = 0; r[1] = -1; r[2] = 0; r[3] = -1; r[4] = 0; r[5] = -1;
        return;
    }
    r[0] = lo[0]; r[1] = hi[0]; r[2] = lo[1]; r[3] = hi[1]; r[4] = lo[2]; r[5] = hi[2];
    const int sy = a.gn[2] + 1, sx = (a.gn[1] + 1) * sy;
    for (int c = 0; c < 8; ++c) {
        int ix = (c & 4) ? hi[0] + 1 : lo[0];
        int iy = (c & 2) ? hi[1] + 1 : lo[1];
        int iz = (c & 1) ? hi[2] + 1 : lo[2];
        int sgn = (__popc(c) & 1) ? -1 : 1;
        atomicAdd(diff + (size_t)ix * sx + (size_t)iy * sy + iz, sgn);
    }
}

// Axis-wise inclusive prefix sums of the (nx+1)(ny+1)(nz+1) difference array.
__global__ void k_prefix_z(int* __restrict__ diff, int nxp, int nyp, int nzp) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nxp * nyp) return;
    int* row = diff + (size_t)t * nzp;
    int s = 0;
    for (int k = 0; k < nzp; ++k) {
        s += row[k];
        row[k] = s;
    }
}

// One warp per line along y (a line is long: 32 of its entries per step, a warp
// scan and a carry).
__global__ void k_prefix_y(int* __restrict__ diff, int nxp, int nyp, int nzp) {
    const int lane = threadIdx.x & 31;
    const long long line = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (line >= (long long)nxp * nzp) return;  // whole warps
    const int i = (int)(line / nzp), k = (int)(line - (long long)i * nzp);
    int* base = diff + (size_t)i * nyp * nzp + k;
    int carry = 0;
    for (int j0 = 0; j0 < nyp; j0 += 32) {
        const int j = j0 + lane;
        int v = j < nyp ? base[(size_t)j * nzp] : 0;
        v = warp_incl_scan(v, lane) + carry;
        if (j < nyp) base[(size_t)j * nzp] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

// Last axis, one warp per line, fused with the write of V_n (dropping the padding
// row of each axis).
__global__ void k_prefix_x(const int* __restrict__ diff, int* __restrict__ v_n, int nx, int ny, int nz) {
    const int lane = threadIdx.x & 31;
    const long long line = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (line >= (long long)ny * nz) return;  // whole warps
    const int j = (int)(line / nz), k = (int)(line - (long long)j * nz);
    const int nzp = nz + 1, nyp = ny + 1;
    int carry = 0;
    for (int i0 = 0; i0 < nx; i0 += 32) {
        const int i = i0 + lane;
        int v = i < nx ? diff[((size_t)i * nyp + j) * nzp + k] : 0;
        v = warp_incl_scan(v, lane) + carry;
        if (i < nx) v_n[((size_t)i * ny + j) * nz + k] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

// -------------------------------------------------------------- exclusive scan
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sh, long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < (blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    long long before = (wid > 0) ? sh[wid - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int* __restrict__ v_n, long long nvox,
                                                              long long* __restrict__ tile_sums) {
    __shared__ long long sh[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < nvox) s += v_n[base + i];
    long long total;
    block_excl_scan(s, sh, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One CTA: exclusive scan of the tile sums (grid-stride over tiles), total P,
// capacity check.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(long long* __restrict__ tile_sums, int n_tiles,
                                                             long long capacity, long long* __restrict__ p_total,
                                                             int* __restrict__ status) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int b = 0; b < n_tiles; b += SCAN_THREADS) {
        int i = b + threadIdx.x;
        long long v = (i < n_tiles) ? tile_sums[i] : 0;
        long long total;
        long long ex = block_excl_scan(v, sh, total);
        if (i < n_tiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        *p_total = carry;
        // SQ_ERR_NUMERIC (set by k_ranges) outranks the capacity error
        if (carry > capacity || carry >= 2147483647LL) atomicMax(status, (int)SQ_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const int* __restrict__ v_n, long long nvox,
                                                             const long long* __restrict__ tile_off,
                                                             int* __restrict__ v_f) {
    __shared__ long long sh[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    int vals[SCAN_ITEMS];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        vals[i] = (base + i < nvox) ? v_n[base + i] : 0;
        s += vals[i];
    }
    long long total;
    long long ex = block_excl_scan(s, sh, total) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < nvox) v_f[base + i] = (int)ex;
        ex += vals[i];
    }
}

// -------------------------------------------------------------- scatter
__global__ void __launch_bounds__(256) k_scatter(const int* __restrict__ ranges, int n, int ny, int nz,
                                                 const int* __restrict__ v_f, int* __restrict__ cursor,
                                                 int* __restrict__ v_sq, long long capacity,
                                                 const int* __restrict__ status) {
    if (*status != SQ_OK) return;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int* r = ranges + 6 * k;
        int dx = r[1] - r[0] + 1, dy = r[3] - r[2] + 1, dz = r[5] - r[4] + 1;
        if (dx <= 0 || dy <= 0 || dz <= 0) continue;
        long long vol = (long long)dx * dy * dz;
        // the thread's voxel of range offset l, advanced by blockDim.x offsets per
        // step as a mixed-radix sum (z fastest): no division inside the loop
        int iz = (int)(threadIdx.x % dz), iy = (int)((threadIdx.x / dz) % dy), ix = (int)(threadIdx.x / dz / dy);
        const int sz = (int)(blockDim.x % dz), syz = (int)(blockDim.x / dz), sy = syz % dy, sx = syz / dy;
        for (long long l = threadIdx.x; l < vol; l += blockDim.x) {
            int v = ((r[0] + ix) * ny + (r[2] + iy)) * nz + (r[4] + iz);
            iz += sz;
            const int cy = iz >= dz ? 1 : 0;
            iz -= cy * dz;
            iy += sy + cy;
            const int cx = iy >= dy ? 1 : 0;
            iy -= cx * dy;
            ix += sx + cx;
            int pos = atomicAdd(cursor + v, 1);
            long long at = (long long)v_f[v] + pos;
            if (at < capacity) v_sq[at] = k;
        }
    }
}

// -------------------------------------------------------------- per-voxel sort
// Ascending bitonic network for any length n: merge steps compare (i, mirror of i)
// then half-cleaners compare (i, i + stride).  Slots >= n act as +inf and are
// never touched (their comparisons cannot swap).
template <typename Load, typename Store>
__device__ void warp_bitonic(int n, int lane, Load ld, Store st) {
    int npow = 1;
    while (npow < n) npow <<= 1;
    const int pairs = npow >> 1;
    for (int size = 2; size <= npow; size <<= 1) {
        const int half = size >> 1;
        for (int t = lane; t < pairs; t += 32) {
            int blk = t / half, pos = t - blk * half;
            int i = blk * size + pos, p = blk * size + size - 1 - pos;
            if (p < n) {
                int a = ld(i), b = ld(p);
                if (a > b) { st(i, b); st(p, a); }
            }
        }
        __syncwarp();
        for (int stride = half >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < pairs; t += 32) {
                int blk = t / stride, pos = t - blk * stride;
                int i = blk * 2 * stride + pos, p = i + stride;
                if (p < n) {
                    int a = ld(i), b = ld(p);
                    if (a > b) { st(i, b); st(p, a); }
                }
            }
            __syncwarp();
        }
    }
}

// Ascending bitonic sort of 32 * E keys held E per lane, element e of lane l
// being key e * 32 + l: compare-exchanges of keys 32 or more apart stay in the
// lane, the others go through shuffles.
template <int E>
__device__ __forceinline__ void reg_bitonic(int (&x)[E], int lane) {
    constexpr int N = 32 * E;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int es = stride >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & es) == 0) {
                        const bool up = ((e * 32 + lane) & size) == 0;
                        const int a = x[e], b = x[e | es];
                        x[e] = up ? min(a, b) : max(a, b);
                        x[e | es] = up ? max(a, b) : min(a, b);
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int y = __shfl_xor_sync(0xffffffffu, x[e], stride);
                    const bool up = ((e * 32 + lane) & size) == 0, lower = (lane & stride) == 0;
                    x[e] = (lower == up) ? min(x[e], y) : max(x[e], y);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void sort_list_regs(int* list, int n, int lane) {
    int x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = e * 32 + lane < n ? list[e * 32 + lane] : 0x7fffffff;
    reg_bitonic<E>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e * 32 + lane < n) list[e * 32 + lane] = x[e];
}

// Range-boundary flags of primitive k listed in voxel (ix, iy, iz): per axis a,
// bit 4a: lo == v, 4a+1: lo == v - 1, 4a+2: hi == v, 4a+3: hi == v + 1.
__device__ __forceinline__ unsigned short entry_flags(const int* __restrict__ ranges, int k, int ix, int iy, int iz) {
    const int* r = ranges + 6 * k;
    const int v[3] = {ix, iy, iz};
    unsigned f = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = __ldg(r + 2 * a), hi = __ldg(r + 2 * a + 1);
        f |= ((lo == v[a]) ? 1u : 0u) << (4 * a);
        f |= ((lo == v[a] - 1) ? 2u : 0u) << (4 * a);
        f |= ((hi == v[a]) ? 4u : 0u) << (4 * a);
        f |= ((hi == v[a] + 1) ? 8u : 0u) << (4 * a);
    }
    return (unsigned short)f;
}

// Sorts every voxel's list ascending (one warp per voxel) and, when v_flags is
// given, writes each entry's range-boundary flags.
__global__ void __launch_bounds__(SORT_WARPS * 32) k_sort(const int* __restrict__ v_n, const int* __restrict__ v_f,
                                                          int* __restrict__ v_sq, long long nvox,
                                                          const int* __restrict__ status,
                                                          const int* __restrict__ ranges,
                                                          unsigned short* __restrict__ v_flags, int ny, int nz) {
    __shared__ int sh[SORT_WARPS][SORT_SMEM];
    if (*status != SQ_OK) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long nwarps = (long long)gridDim.x * SORT_WARPS;
    for (long long v = (long long)blockIdx.x * SORT_WARPS + wid; v < nvox; v += nwarps) {
        const int n = v_n[v];
        if (n < 1) continue;
        int* list = v_sq + v_f[v];
        if (n == 1) {
            // a single entry is sorted
        } else if (n <= 32) {
            sort_list_regs<1>(list, n, lane);
        } else if (n <= 64) {
            sort_list_regs<2>(list, n, lane);
        } else if (n <= 128) {
            sort_list_regs<4>(list, n, lane);
        } else if (n <= 256) {
            sort_list_regs<8>(list, n, lane);
        } else if (n <= SORT_SMEM) {
            int* s = sh[wid];
            for (int i = lane; i < n; i += 32) s[i] = list[i];
            __syncwarp();
            warp_bitonic(n, lane, [&](int i) { return s[i]; }, [&](int i, int val) { s[i] = val; });
            for (int i = lane; i < n; i += 32) list[i] = s[i];
            __syncwarp();
        } else {
            volatile int* g = list;
            warp_bitonic(n, lane, [&](int i) { return g[i]; }, [&](int i, int val) { g[i] = val; });
        }
        if (v_flags) {
            __syncwarp();
            const int iz = (int)(v % nz), iy = (int)((v / nz) % ny), ix = (int)(v / ((long long)ny * nz));
            unsigned short* fl = v_flags + v_f[v];
            for (int i = lane; i < n; i += 32) fl[i] = entry_flags(ranges, list[i], ix, iy, iz);
        }
    }
}

// -------------------------------------------------------------- lists by voxel tiles
// V_sq without atomics or a sort: a block takes a tile of LT_X x LT_Y x LT_Z voxels,
// one voxel per thread, and scans the packed voxel ranges in id order (rounds of
// LT_ROUND ids, warp w the w-th window of LT_WIN ids, the warps' hits in warp
// order being the round's hits in id order), each hit with the tile-local bit
// masks of its x, y and z extent.  Every thread then walks the held hits (up to
// LT_CAP, several rounds') and appends those whose range holds its voxel to the
// voxel's list: the list is written in ascending id, exactly the sorted list of
// the primitives whose range contains the voxel.  Each warp holds a 4 x 4 x 2
// block of the tile.
constexpr int LT_X = 8, LT_Y = 8, LT_Z = 4, LT_THREADS = LT_X * LT_Y * LT_Z;
constexpr int LT_WIN = 128, LT_ROUND = LT_WIN * (LT_THREADS / 32);
constexpr int LT_CAP = 2 * LT_ROUND;  // hits held before the voxels append them (a round adds at most LT_ROUND)
static_assert(LT_THREADS == 256, "warps of 4 x 4 x 2 voxels");

__device__ __forceinline__ unsigned lt_span(int lo, int hi) { return hi < lo ? 0u : (2u << hi) - (1u << lo); }

__global__ void __launch_bounds__(LT_THREADS) k_lists_tiles(const int4* __restrict__ boxes, int n,
                                                           const int* __restrict__ v_f, int* __restrict__ v_sq,
                                                           long long capacity, const int* __restrict__ status,
                                                           const int* __restrict__ ranges,
                                                           unsigned short* __restrict__ v_flags, int nx, int ny,
                                                           int nz, int ntx, int nty, int ntz) {
    __shared__ int wid_[LT_THREADS / 32][LT_WIN];
    __shared__ unsigned wmsk[LT_THREADS / 32][LT_WIN];
    __shared__ int lid[LT_CAP];
    __shared__ unsigned lmsk[LT_CAP];
    __shared__ int wtot[LT_THREADS / 32];
    if (*status != SQ_OK) return;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int lx = (wid & 1) * 4 + (lane & 3), ly = ((wid >> 1) & 1) * 4 + ((lane >> 2) & 3),
              lz = (wid >> 2) * 2 + (lane >> 4);
    const unsigned sel = (1u << lx) | (1u << (8 + ly)) | (1u << (16 + lz));
    for (int tile = blockIdx.x; tile < ntx * nty * ntz; tile += gridDim.x) {
        const int tz = tile % ntz, ty = (tile / ntz) % nty, tx = tile / (ntz * nty);
        const int x0 = tx * LT_X, y0 = ty * LT_Y, z0 = tz * LT_Z;
        const int x1 = min(x0 + LT_X, nx) - 1, y1 = min(y0 + LT_Y, ny) - 1, z1 = min(z0 + LT_Z, nz) - 1;
        const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
        const bool valid = ix <= x1 && iy <= y1 && iz <= z1;
        const long long v = valid ? ((long long)ix * ny + iy) * nz + iz : 0;
        const long long vf = valid ? (long long)__ldg(v_f + v) : 0;
        int cnt = 0;
        int base = 0;  // hits held in lid / lmsk (the same in every thread)
        for (int r0 = 0; r0 < n; r0 += LT_ROUND) {
            int wc = 0;
#pragma unroll
            for (int s2 = 0; s2 < LT_WIN / 32; ++s2) {
                const int k = r0 + wid * LT_WIN + s2 * 32 + lane;
                unsigned m = 0u;
                if (k < n) {
                    const int4 b = __ldg(boxes + k);
                    const int bx0 = b.x & 0xffff, bx1 = (int)((unsigned)b.x >> 16);
                    const int by0 = b.y & 0xffff, by1 = (int)((unsigned)b.y >> 16);
                    const int bz0 = b.z & 0xffff, bz1 = (int)((unsigned)b.z >> 16);
                    if (bx0 <= x1 && bx1 >= x0 && by0 <= y1 && by1 >= y0 && bz0 <= z1 && bz1 >= z0 &&
                        bx0 <= bx1 && by0 <= by1 && bz0 <= bz1)
                        m = lt_span(max(bx0, x0) - x0, min(bx1, x1) - x0) |
                            (lt_span(max(by0, y0) - y0, min(by1, y1) - y0) << 8) |
                            (lt_span(max(bz0, z0) - z0, min(bz1, z1) - z0) << 16);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, m != 0u);
                if (m != 0u) {
                    const int pos = wc + __popc(bal & ((1u << lane) - 1u));
                    wid_[wid][pos] = k;
                    wmsk[wid][pos] = m;
                }
                wc += __popc(bal);
            }
            if (lane == 0) wtot[wid] = wc;
            __syncthreads();
            int before = 0, nc = 0;
#pragma unroll
            for (int w2 = 0; w2 < LT_THREADS / 32; ++w2) {
                const int c = wtot[w2];
                before += w2 < wid ? c : 0;
                nc += c;
            }
            for (int j = lane; j < wc; j += 32) {
                lid[base + before + j] = wid_[wid][j];
                lmsk[base + before + j] = wmsk[wid][j];
            }
            base += nc;
            __syncthreads();
            // the held hits, in id order, once the buffer could not take another round
            if (base > LT_CAP - LT_ROUND || r0 + LT_ROUND >= n) {
                for (int j = 0; j < base; ++j) {
                    if ((lmsk[j] & sel) == sel) {  // only valid voxels have their bits set
                        const long long at = vf + cnt;
                        const int k = lid[j];
                        if (at < capacity) {
                            v_sq[at] = k;
                            if (v_flags) v_flags[at] = entry_flags(ranges, k, ix, iy, iz);
                        }
                        ++cnt;
                    }
                }
                base = 0;
                __syncthreads();
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- workspace
struct IndexWs {
    size_t diff_off, cursor_off, tiles_off, total;
};

static IndexWs index_ws(const sq_grid_t* g) {
    IndexWs w;
    size_t ndiff = (size_t)(g->nx + 1) * (g->ny + 1) * (g->nz + 1);
    size_t nvox = (size_t)g->nx * g->ny * g->nz;
    size_t ntiles = (nvox + SCAN_TILE - 1) / SCAN_TILE;
    w.diff_off = 0;
    w.cursor_off = align_up(w.diff_off + ndiff * sizeof(int), 256);
    w.tiles_off = align_up(w.cursor_off + nvox * sizeof(int), 256);
    w.total = align_up(w.tiles_off + ntiles * sizeof(long long), 256);
    return w;
}

size_t index_workspace_size(const sq_grid_t* g) { return index_ws(g).total; }

sq_status_t build_index_impl(const sq_prims_t* prims, const sq_grid_t* grid, const sq_index_opts_t* opts,
                             sq_index_t* idx, void* ws, size_t ws_bytes, cudaStream_t st) {
    IndexWs w = index_ws(grid);
    if (ws_bytes < w.total || (w.total > 0 && ws == nullptr)) {
        set_last_error("sq_build_index: workspace of %zu bytes given, %zu needed", ws_bytes, w.total);
        return SQ_ERR_INVALID_ARG;
    }
    char* base = (char*)ws;
    int* diff = (int*)(base + w.diff_off);
    int* cursor = (int*)(base + w.cursor_off);
    long long* tiles = (long long*)(base + w.tiles_off);
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    const long long nvox = (long long)nx * ny * nz;
    const size_t ndiff = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    const int n_tiles = (int)((nvox + SCAN_TILE - 1) / SCAN_TILE);

    // The lists are built by voxel tiles when the ranges pack into 16 bits per end
    // and the packed ranges fit in the cursor block (which that build does not use);
    // otherwise by the scatter and the per-voxel sort.
    const bool by_tiles = nx <= 65535 && ny <= 65535 && nz <= 65535 && prims->n > 0 &&
                          (size_t)prims->n * sizeof(int4) <= (size_t)nvox * sizeof(int);
    cudaError_t e;
    e = cudaMemsetAsync(diff, 0, ndiff * sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e, "memset diff");
    if (!by_tiles) {
        e = cudaMemsetAsync(cursor, 0, (size_t)nvox * sizeof(int), st);
        if (e != cudaSuccess) return cuda_status(e, "memset cursor");
    }
    e = cudaMemsetAsync(idx->status, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e, "memset status");

    RangeArgs a;
    a.means = prims->means; a.quats = prims->quats; a.scales = prims->scales; a.eps = prims->eps;
    a.opacity = prims->opacity;
    a.logits = prims->logits;
    a.C = prims->n_classes;
    a.status = idx->status;
    a.n = prims->n; a.mode = opts->mode; a.nv = opts->nv;
    a.log_kc = (opts->mode != SQ_INDEX_CUBE) ? log(-log((double)opts->tau_cut)) : 0.0;
    a.tau = (double)opts->tau_cut;
    a.log_tau = log((double)opts->tau_cut);
    a.gn[0] = nx; a.gn[1] = ny; a.gn[2] = nz;
    for (int i = 0; i < 3; ++i) { a.glo[i] = grid->lo[i]; a.gvs[i] = grid->vs[i]; }

    if (prims->n > 0) {
        SQ_LAUNCH("k_ranges", st, k_ranges<<<(prims->n + 127) / 128, 128, 0, st>>>(a, idx->ranges, diff));
    }
    const int nxp = nx + 1, nyp = ny + 1, nzp = nz + 1;
    SQ_LAUNCH("k_prefix_z", st, k_prefix_z<<<(nxp * nyp + 255) / 256, 256, 0, st>>>(diff, nxp, nyp, nzp));
    SQ_LAUNCH("k_prefix_y", st, k_prefix_y<<<(unsigned)(((long long)nxp * nzp * 32 + 255) / 256), 256, 0, st>>>(diff, nxp, nyp, nzp));
    SQ_LAUNCH("k_prefix_x", st, k_prefix_x<<<(unsigned)(((long long)ny * nz * 32 + 255) / 256), 256, 0, st>>>(diff, idx->v_n, nx, ny, nz));
    SQ_LAUNCH("k_scan_reduce", st, k_scan_reduce<<<n_tiles, SCAN_THREADS, 0, st>>>(idx->v_n, nvox, tiles));
    SQ_LAUNCH("k_scan_tiles", st, k_scan_tiles<<<1, SCAN_THREADS, 0, st>>>(tiles, n_tiles, idx->capacity, idx->p_total, idx->status));
    SQ_LAUNCH("k_scan_apply", st, k_scan_apply<<<n_tiles, SCAN_THREADS, 0, st>>>(idx->v_n, nvox, tiles, idx->v_f));
    if (by_tiles) {
        int4* boxes = reinterpret_cast<int4*>(cursor);  // 16-byte aligned (a 256-byte aligned block)
        sq_status_t sb = launch_pack_boxes(idx->ranges, prims->n, boxes, st);
        if (sb != SQ_OK) return sb;
        const int ntx = (nx + LT_X - 1) / LT_X, nty = (ny + LT_Y - 1) / LT_Y, ntz = (nz + LT_Z - 1) / LT_Z;
        const long long ntl = (long long)ntx * nty * ntz;
        const int lblocks = (int)(ntl < (1LL << 30) ? ntl : (1LL << 30));
        SQ_LAUNCH("k_lists_tiles", st,
                  k_lists_tiles<<<lblocks, LT_THREADS, 0, st>>>(boxes, prims->n, idx->v_f, idx->v_sq, idx->capacity,
                                                                idx->status, idx->ranges, idx->v_flags, nx, ny, nz,
                                                                ntx, nty, ntz));
    } else if (prims->n > 0) {
        int blocks = prims->n < 65535 ? prims->n : 65535;
        SQ_LAUNCH("k_scatter", st, k_scatter<<<blocks, 256, 0, st>>>(idx->ranges, prims->n, ny, nz, idx->v_f, cursor, idx->v_sq, idx->capacity,
                                          idx->status));
        long long want = (nvox + SORT_WARPS - 1) / SORT_WARPS;
        int sblocks = (int)(want < 152 * 64 ? want : 152 * 64);
        SQ_LAUNCH("k_sort", st, k_sort<<<sblocks, SORT_WARPS * 32, 0, st>>>(idx->v_n, idx->v_f, idx->v_sq, nvox, idx->status, idx->ranges,
                                                    idx->v_flags, ny, nz));
    }
    return SQ_OK;
}

}  // namespace sqr
