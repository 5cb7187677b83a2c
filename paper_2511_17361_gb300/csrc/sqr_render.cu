// sqr_render.cu -- host side of the renderer: packing of the superquadric
// parameters into the kernels' records, workspace layout, the single-scene and
// batched forward/backward calls (one persistent launch over the rays of every
// scene), the launch-configuration autotuner, and the pair counter.
#include <math.h>
#include <string.h>

#include "sqr_render.cuh"

namespace sqr {

namespace {

// ------------------------------------------------------------------ packing
// Forward record (4 x float4): (m, sigma), (M_0, ea), (M_1, eb), (M_2, ec) with
// M_j = (column j of R(q/|q|)) / s_j, ea = 2/eps2, eb = eps2/eps1, ec = 2/eps1.
// Backward extras (3 x float4): (qn), (1/|q|, 1/s), (eps1, eps2, 1/eps1, 1/eps2).
__global__ void k_pack(sq_prims_t P, float4* __restrict__ rec, float4* __restrict__ aux, float* __restrict__ lpad,
                       int cp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n) return;
    // In FP64, each packed value rounded to FP32 once: the scaled coordinate
    // u_j = M_j . (x - m) cancels near the planes u_j = 0 of the primitive's frame,
    // where df/dx holds |u_j|^(2/eps - 1); an M carrying the roundings of an FP32
    // construction cost the gradient there two decimal digits.
    double w = P.quats[4 * k + 0], x = P.quats[4 * k + 1], y = P.quats[4 * k + 2], z = P.quats[4 * k + 3];
    const double nq = sqrt(w * w + x * x + y * y + z * z);
    const double inq = 1.0 / nq;
    w *= inq; x *= inq; y *= inq; z *= inq;
    double R[3][3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z); R[0][1] = 2.0 * (x * y - w * z); R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z); R[1][1] = 1.0 - 2.0 * (x * x + z * z); R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y); R[2][1] = 2.0 * (y * z + w * x); R[2][2] = 1.0 - 2.0 * (x * x + y * y);
    const double is[3] = {1.0 / P.scales[3 * k + 0], 1.0 / P.scales[3 * k + 1], 1.0 / P.scales[3 * k + 2]};
    const double e1 = P.eps[2 * k + 0], e2 = P.eps[2 * k + 1];
    float M[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) M[j][i] = (float)(R[i][j] * is[j]);
    float4* r = rec + (size_t)k * REC4;
    r[0] = make_float4(P.means[3 * k + 0], P.means[3 * k + 1], P.means[3 * k + 2], P.opacity[k]);
    r[1] = make_float4(M[0][0], M[0][1], M[0][2], (float)(2.0 / e2));
    r[2] = make_float4(M[1][0], M[1][1], M[1][2], (float)(e2 / e1));
    r[3] = make_float4(M[2][0], M[2][1], M[2][2], (float)(2.0 / e1));
    if (aux) {
        float4* a = aux + (size_t)k * AUX4;
        a[0] = make_float4((float)w, (float)x, (float)y, (float)z);
        a[1] = make_float4((float)inq, (float)is[0], (float)is[1], (float)is[2]);
        a[2] = make_float4((float)e1, (float)e2, (float)(1.0 / e1), (float)(1.0 / e2));
    }
    const int C = P.n_classes;
    const float* lg = P.logits + (size_t)k * C;
    if (P.sem_mode == SQ_SEM_SOFTMAX) {  // per-primitive softmax of the logits
        float mx = lg[0];
        for (int c = 1; c < C; ++c) mx = fmaxf(mx, lg[c]);
        float sum = 0.f;
        for (int c = 0; c < C; ++c) sum += expf(lg[c] - mx);
        const float inv = 1.0f / sum;
        for (int c = 0; c < cp; ++c) lpad[(size_t)k * cp + c] = c < C ? expf(lg[c] - mx) * inv : 0.f;
    } else {
        for (int c = 0; c < cp; ++c) lpad[(size_t)k * cp + c] = c < C ? lg[c] : 0.f;
    }
}

// Copies the by-value scene descriptors into device memory (one thread).
__global__ void k_write_desc(BatchParams P, SceneDesc* __restrict__ d, long long* __restrict__ off,
                             long long* __restrict__ boff, long long* __restrict__ gboff,
                             long long* __restrict__ poff) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < P.n; ++i) d[i] = P.s[i];
    long long np = 0;
    for (int i = 0; i <= P.n; ++i) {
        off[i] = P.off[i];
        boff[i] = P.boff[i];
        poff[i] = np;
        if (i < P.n) np += P.s[i].n;
    }
    for (int i = 0; i < 2 * MAX_BATCH; ++i) gboff[i] = P.gboff[i];
}

// ------------------------------------------------------------------ pair counter
__global__ void __launch_bounds__(256) k_count_pairs(SceneDesc S, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long sq[8], ss[8];
    unsigned long long q = 0, s = 0;
    const long long total = S.R * S.L;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / S.L;
        const int j = (int)(e - r * S.L);
        float o[3], d[3], x[3];
        scene_ray(S, r, o, d);
        const int vox = sample_voxel(S.g, o, d, __ldg(S.t + j), x);
        if (vox >= 0) {
            q += (unsigned long long)__ldg(S.v_n + vox);
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

// ------------------------------------------------------------------ workspace
// Header: descriptors, ray offsets, work counter.  Then per scene: forward
// records, backward extras, padded logits, gradient accumulator, packed boxes.
struct SceneWs {
    size_t rec, aux, lpad, gacc, box, end;
};

constexpr size_t HDR_DESC = 0;
constexpr size_t HDR_OFF = (MAX_BATCH * sizeof(SceneDesc) + 255) / 256 * 256;
constexpr size_t HDR_BOFF = HDR_OFF + ((MAX_BATCH + 1) * sizeof(long long) + 255) / 256 * 256;
constexpr size_t HDR_GBOFF = HDR_BOFF + ((MAX_BATCH + 1) * sizeof(long long) + 255) / 256 * 256;
constexpr size_t HDR_POFF = HDR_GBOFF + (2 * MAX_BATCH * sizeof(long long) + 255) / 256 * 256;
constexpr size_t HDR_CTR = HDR_POFF + ((MAX_BATCH + 1) * sizeof(long long) + 255) / 256 * 256;
constexpr size_t HDR_END = HDR_CTR + 256;
constexpr int CTR_PM = 48;  // counter of the primitive-major tile walk (slots 0..MAX_BATCH serve the others)

SceneWs scene_ws(const sq_prims_t* p, size_t base) {
    SceneWs w;
    const size_t n = (size_t)(p->n > 0 ? p->n : 0);
    const int cp = cpad(p->n_classes);
    w.rec = align_up(base, 256);
    w.aux = align_up(w.rec + n * REC4 * sizeof(float4), 256);
    w.lpad = align_up(w.aux + n * AUX4 * sizeof(float4), 256);
    w.gacc = align_up(w.lpad + n * cp * sizeof(float), 256);
    w.box = align_up(w.gacc + n * GF * sizeof(float), 256);
    w.end = align_up(w.box + n * sizeof(int4), 256);
    return w;
}

// The backward's per-sample (dL/dalpha_j, w_j) of every scene follow the scene
// blocks, so a forward needs only the prefix; then the primitive-major
// backward's blocks: per scene the box rectangles [n, n_cam], and over all
// primitives the candidate counts, tile offsets and tile sums.
size_t gw_bytes(const sq_rays_t* r) { return align_up((size_t)r->n_cam * r->H * r->W * r->L * sizeof(float2), 256); }

size_t rect_bytes(const sq_scene_t* s) {
    return align_up((size_t)(s->prims.n > 0 ? s->prims.n : 0) * (size_t)(s->rays.n_cam > 0 ? s->rays.n_cam : 0) *
                        sizeof(int4),
                    256);
}

size_t dir_bytes(const sq_rays_t* r) { return align_up((size_t)r->n_cam * r->H * r->W * sizeof(float4), 256); }

size_t gs_bytes(const sq_rays_t* r, int C) {
    return align_up((size_t)r->n_cam * r->H * r->W * (size_t)cpad(C) * sizeof(float), 256);
}

struct PmWs {
    size_t cnt, toff, tprim, part, key, qtile, end;
};

PmWs pm_ws(size_t at, long long ntot) {
    PmWs w;
    w.cnt = align_up(at, 256);
    w.toff = align_up(w.cnt + (size_t)ntot * sizeof(int), 256);
    w.tprim = align_up(w.toff + (size_t)(ntot + 1) * sizeof(int), 256);
    w.part = align_up(w.tprim + (size_t)ntot * PM_MAXT * sizeof(int), 256);
    w.key = align_up(w.part + (size_t)ntot * PM_MAXT * GF * sizeof(float), 256);
    w.qtile = align_up(w.key + (size_t)ntot * sizeof(int), 256);
    w.end = align_up(w.qtile + (size_t)ntot * PM_MAXT * sizeof(int), 256);
    return w;
}

size_t batch_ws_size(const sq_scene_t* sc, int n, bool bwd) {
    size_t at = HDR_END;
    for (int i = 0; i < n; ++i) at = scene_ws(&sc[i].prims, at).end;
    if (bwd) {
        long long ntot = 0;
        for (int i = 0; i < n; ++i) {
            at += gw_bytes(&sc[i].rays);
            at += rect_bytes(&sc[i]);
            at += dir_bytes(&sc[i].rays);
            at += gs_bytes(&sc[i].rays, sc[i].prims.n_classes);
            ntot += sc[i].prims.n > 0 ? sc[i].prims.n : 0;
        }
        at = pm_ws(at, ntot).end;
    }
    return at;
}

// Saved forward state (sq_saved_size): a 256-byte header (int64 pages needed,
// int32 status), the page of every SAVE_PS samples of every ray [R, ceil(L /
// SAVE_PS)] int32, the composited count [R] int32, then cap pages of SAVE_PS
// samples: (T, signed alpha) float2 each, and s [CP] float each (CP = C rounded
// up to 4, zero-padded).  Each block 256-byte aligned.
constexpr size_t SAVE_HDR = 256;

size_t saved_fixed_bytes(const sq_rays_t* r) {
    const size_t R = (size_t)r->n_cam * r->H * r->W, np = ((size_t)r->L + SAVE_PS - 1) / SAVE_PS;
    return SAVE_HDR + align_up(R * np * sizeof(int), 256) + align_up(R * sizeof(int), 256);
}

size_t saved_bytes_pages(const sq_rays_t* r, int C, long long pages) {
    const size_t ns = (size_t)(pages > 0 ? pages : 0) * SAVE_PS;
    return saved_fixed_bytes(r) + align_up(ns * sizeof(float2), 256) + align_up(ns * (size_t)cpad(C) * sizeof(float), 256);
}

// Pages that every sample of every ray needs at most.
long long saved_pages_max(const sq_rays_t* r) {
    return (long long)r->n_cam * r->H * r->W * (((long long)r->L + SAVE_PS - 1) / SAVE_PS);
}

size_t saved_bytes_of(const sq_rays_t* r, int C) { return saved_bytes_pages(r, C, saved_pages_max(r)); }

// Pages a buffer of `bytes` holds (0 if it cannot hold the fixed blocks).
long long saved_cap_of(const sq_rays_t* r, int C, size_t bytes) {
    const size_t fixed = saved_fixed_bytes(r);
    if (bytes <= fixed) return 0;
    const size_t per = SAVE_PS * (sizeof(float2) + (size_t)cpad(C) * sizeof(float));
    long long cap = (long long)((bytes - fixed) / per);  // the two blocks' alignment takes at most 510 bytes
    while (cap > 0 && saved_bytes_pages(r, C, cap) > bytes) --cap;
    return cap;
}

void saved_ptrs(const sq_rays_t* r, int C, void* saved, size_t bytes, SceneDesc& D) {
    const size_t R = (size_t)r->n_cam * r->H * r->W, np = ((size_t)r->L + SAVE_PS - 1) / SAVE_PS;
    const long long cap = saved_cap_of(r, C, bytes);
    char* p = (char*)saved;
    D.save_ctr = (unsigned long long*)p;
    D.save_status = (int*)(p + 8);
    p += SAVE_HDR;
    D.save_page = (int*)p;
    p += align_up(R * np * sizeof(int), 256);
    D.save_n = (int*)p;
    p += align_up(R * sizeof(int), 256);
    D.save_TA = (float2*)p;
    p += align_up((size_t)cap * SAVE_PS * sizeof(float2), 256);
    D.save_S = (float4*)p;
    D.save_cap = cap;
    D.save_np = (int)np;
}

Tuning default_tuning() { return Tuning{4, 8, 0, SQ_BWD_PRIMITIVE_MAJOR, 1}; }

}  // namespace

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
    return sms;
}

sq_status_t launch_pack(const sq_prims_t* prims, float4* rec, float4* aux, float* lpad, int cp, cudaStream_t st) {
    if (prims->n == 0) return SQ_OK;
    SQ_LAUNCH("k_pack", st, k_pack<<<(prims->n + 127) / 128, 128, 0, st>>>(*prims, rec, aux, lpad, cp));
    return SQ_OK;
}

size_t saved_size(const sq_rays_t* r, int n_classes) { return saved_bytes_of(r, n_classes); }

size_t saved_size_pages(const sq_rays_t* r, int n_classes, long long pages) {
    return saved_bytes_pages(r, n_classes, pages);
}

size_t batched_workspace_size(const sq_scene_t* scenes, int n) {
    bool train = n > 0;
    for (int i = 0; i < n; ++i) train = train && scenes[i].saved != nullptr;
    return batch_ws_size(scenes, n, train);
}

size_t render_workspace_size(const sq_prims_t* p) {
    sq_scene_t s;
    memset(&s, 0, sizeof(s));
    s.prims = *p;
    return batch_ws_size(&s, 1, false);
}

size_t render_bwd_workspace_size(const sq_prims_t* p, const sq_rays_t* r) {
    sq_scene_t s;
    memset(&s, 0, sizeof(s));
    s.prims = *p;
    s.rays = *r;
    return batch_ws_size(&s, 1, true);
}

// Validates a batch for op, packs every scene, writes the descriptors and runs
// the persistent forward or backward launch over all rays of all scenes.
sq_status_t batched_impl(int op, const sq_scene_t* sc, int n, const Tuning& tn, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
    if (n < 1 || n > MAX_BATCH) {
        set_last_error("batch of %d scenes, 1..%d supported", n, MAX_BATCH);
        return SQ_ERR_INVALID_ARG;
    }
    const size_t need = batch_ws_size(sc, n, op == SQ_OP_BWD);
    if (ws == nullptr || ws_bytes < need) {
        set_last_error("render workspace of %zu bytes given, %zu needed", ws_bytes, need);
        return SQ_ERR_INVALID_ARG;
    }
    const int C = sc[0].prims.n_classes, cp = cpad(C);
    BatchParams P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    char* base = (char*)ws;
    long long total = 0, btotal = 0;
    const int RB = bwd_rays_per_bundle();
    int lmax = 0;
    size_t at = HDR_END;
    for (int i = 0; i < n; ++i) {
        const sq_scene_t& s = sc[i];
        if (s.prims.n_classes != C) {
            set_last_error("all scenes of a batch need the same n_classes (%d vs %d)", s.prims.n_classes, C);
            return SQ_ERR_INVALID_ARG;
        }
        const long long R = (long long)s.rays.n_cam * s.rays.H * s.rays.W;
        if (op == SQ_OP_FWD && R > 0 && (!s.depth || !s.sem)) {
            set_last_error("scene %d: depth/sem output is NULL", i);
            return SQ_ERR_INVALID_ARG;
        }
        const size_t sneed = saved_bytes_pages(&s.rays, C, 1);  // the fixed blocks and one page
        if (op == SQ_OP_FWD && s.saved && s.saved_bytes < sneed) {
            set_last_error("scene %d: saved state of %zu bytes given, at least %zu needed", i, s.saved_bytes, sneed);
            return SQ_ERR_INVALID_ARG;
        }
        if (op == SQ_OP_BWD) {
            if (!s.saved || s.saved_bytes < sneed) {
                set_last_error("scene %d: backward needs the saved forward state (%zu bytes given, at least %zu)", i,
                               s.saved_bytes, sneed);
                return SQ_ERR_INVALID_ARG;
            }
            if (R > 0 && (!s.grad_depth || !s.grad_sem)) {
                set_last_error("scene %d: grad_depth/grad_sem is NULL", i);
                return SQ_ERR_INVALID_ARG;
            }
            if (s.prims.n > 0 &&
                (!s.g_means || !s.g_quats || !s.g_scales || !s.g_eps || !s.g_opacity || !s.g_logits)) {
                set_last_error("scene %d: a gradient output is NULL", i);
                return SQ_ERR_INVALID_ARG;
            }
            if (s.grid.nx > 65535 || s.grid.ny > 65535 || s.grid.nz > 65535) {
                set_last_error("scene %d: backward supports grid dims up to 65535 per axis", i);
                return SQ_ERR_INVALID_ARG;
            }
        }
        const SceneWs w = scene_ws(&s.prims, at);
        at = w.end;
        SceneDesc& D = P.s[i];
        D.rec = (const float4*)(base + w.rec);
        D.aux = (const float4*)(base + w.aux);
        D.lpad = (const float*)(base + w.lpad);
        D.boxes = (const int4*)(base + w.box);
        D.v_n = s.index.v_n;
        D.v_f = s.index.v_f;
        D.v_sq = s.index.v_sq;
        D.v_cap = s.index.capacity;
        D.v_flags = s.index.v_flags;
        D.status = s.index.status;
        D.g = make_grid(&s.grid);
        D.K = s.rays.K;
        D.c2w = s.rays.cam2world;
        D.t = s.rays.t;
        D.n_cam = s.rays.n_cam;
        D.H = s.rays.H;
        D.W = s.rays.W;
        D.L = s.rays.L;
        D.C = C;
        D.n = s.prims.n;
        D.sem_mode = s.prims.sem_mode;
        D.cp = cp;
        D.R = R;
        D.kappa = s.rays.kappa;
        D.alpha_max = s.rays.alpha_max;
        D.depth = s.depth;
        D.sem = s.sem;
        D.t_final = s.t_final;
        if (s.saved) {
            saved_ptrs(&s.rays, C, s.saved, s.saved_bytes, D);
            if (op == SQ_OP_FWD) {  // page counter and status start at zero
                cudaError_t e = cudaMemsetAsync(s.saved, 0, 16, st);
                if (e != cudaSuccess) return cuda_status(e, "memset saved header");
            }
        }
        D.grad_depth = s.grad_depth;
        D.grad_sem = s.grad_sem;
        D.pair_visits = s.pair_visits;
        D.gacc = (float*)(base + w.gacc);
        P.off[i] = total;
        P.boff[i] = btotal;
        total += R;
        btotal += (R + RB - 1) / RB;
        if (s.rays.L > lmax) lmax = s.rays.L;
        if (total >= 2147483647LL - 4096) {
            set_last_error("a batch holds at most 2^31 - 4096 rays");
            return SQ_ERR_INVALID_ARG;
        }
        sq_status_t ps = launch_pack(&s.prims, (float4*)(base + w.rec), (float4*)(base + w.aux),
                                     (float*)(base + w.lpad), cp, st);
        if (ps != SQ_OK) return ps;
        if (op == SQ_OP_BWD && s.prims.n > 0) {
            cudaError_t e = cudaMemsetAsync(base + w.gacc, 0, (size_t)s.prims.n * GF * sizeof(float), st);
            if (e != cudaSuccess) return cuda_status(e, "memset gradient accumulator");
            ps = launch_pack_boxes(s.index.ranges, s.prims.n, (int4*)(base + w.box), st);
            if (ps != SQ_OK) return ps;
        }
    }
    P.off[n] = total;
    P.boff[n] = btotal;
    // backward launch groups: consecutive scenes of equal L (the run walk sizes each
    // warp's sample table by the launch's largest L); group g's bundle offsets sit at
    // gboff[i0 + g ..], counted from its first scene i0
    int gfirst[MAX_BATCH + 1], ng = 0;
    for (int i0 = 0; i0 < n;) {
        int i1 = i0 + 1;
        while (i1 < n && sc[i1].rays.L == sc[i0].rays.L) ++i1;
        for (int i = i0; i <= i1; ++i) P.gboff[i + ng] = P.boff[i] - P.boff[i0];
        gfirst[ng++] = i0;
        i0 = i1;
    }
    gfirst[ng] = n;
    long long ntot = 0;
    PmWs pw{};
    if (op == SQ_OP_BWD) {
        for (int i = 0; i < n; ++i) {
            P.s[i].gw = (float2*)(base + at);
            at += gw_bytes(&sc[i].rays);
            P.s[i].pm_rect = (int4*)(base + at);
            at += rect_bytes(&sc[i]);
            P.s[i].pm_dir = (float4*)(base + at);
            at += dir_bytes(&sc[i].rays);
            P.s[i].pm_gs = (float4*)(base + at);
            at += gs_bytes(&sc[i].rays, C);
            ntot += sc[i].prims.n;
        }
        if (ntot * PM_MAXT >= 2147483647LL) {
            set_last_error("a backward batch holds at most %d primitives", (int)(2147483647LL / PM_MAXT));
            return SQ_ERR_INVALID_ARG;
        }
        pw = pm_ws(at, ntot);
    }
    SceneDesc* d = (SceneDesc*)(base + HDR_DESC);
    long long* off = (long long*)(base + HDR_OFF);
    long long* boff = (long long*)(base + HDR_BOFF);
    long long* gboff = (long long*)(base + HDR_GBOFF);
    long long* poff = (long long*)(base + HDR_POFF);
    int* ctr = (int*)(base + HDR_CTR);
    SQ_LAUNCH("k_write_desc", st, k_write_desc<<<1, 32, 0, st>>>(P, d, off, boff, gboff, poff));
    cudaError_t e = cudaMemsetAsync(ctr, 0, 256, st);
    if (e != cudaSuccess) return cuda_status(e, "memset counter");
    Batch B{d, off, boff, n, total, ctr, lmax, tn.fwd_tile};
    sq_status_t ls = (op == SQ_OP_FWD) ? launch_forward(B, cp, tn, st) : launch_sweep(B, cp, st);
    if (ls != SQ_OK) return ls;
    if (op == SQ_OP_BWD) {
        if (tn.bwd_order == SQ_BWD_PRIMITIVE_MAJOR) {
            const PmArgs A{poff,
                           n,
                           (int)ntot,
                           (int*)(base + pw.cnt),
                           (int*)(base + pw.toff),
                           (float*)(base + pw.part),
                           (int*)(base + pw.tprim),
                           ctr + CTR_PM,
                           (int*)(base + pw.key),
                           (int*)(base + pw.qtile)};
            ls = launch_backward_pm(B, A, cp, st);
            if (ls != SQ_OK) return ls;
        } else {
            for (int g = 0; g < ng; ++g) {  // one run-walk launch per group, each with its own counter
                const int i0 = gfirst[g], i1 = gfirst[g + 1];
                const Batch Bg{d + i0, off + i0, gboff + i0 + g, i1 - i0, P.off[i1] - P.off[i0], ctr + 1 + g,
                               sc[i0].rays.L};
                ls = launch_backward(Bg, cp, tn, st);
                if (ls != SQ_OK) return ls;
            }
        }
        for (int i = 0; i < n; ++i) {
            const sq_scene_t& s = sc[i];
            ls = launch_grad_out(P.s[i], s.g_means, s.g_quats, s.g_scales, s.g_eps, s.g_opacity, s.g_logits, st);
            if (ls != SQ_OK) return ls;
        }
    }
    return SQ_OK;
}

sq_status_t render_fwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* saved,
                            size_t saved_bytes, void* ws, size_t ws_bytes, cudaStream_t st) {
    sq_scene_t s;
    memset(&s, 0, sizeof(s));
    s.prims = *prims;
    s.index = *idx;
    s.grid = *grid;
    s.rays = *rays;
    s.depth = depth;
    s.sem = sem;
    s.t_final = t_final;
    s.saved = saved;
    s.saved_bytes = saved_bytes;
    return batched_impl(SQ_OP_FWD, &s, 1, default_tuning(), ws, ws_bytes, st);
}

sq_status_t render_bwd_impl(const sq_prims_t* prims, const sq_index_t* idx, const sq_grid_t* grid,
                            const sq_rays_t* rays, const void* saved, size_t saved_bytes, const float* grad_depth,
                            const float* grad_sem, float* g_means, float* g_quats, float* g_scales, float* g_eps,
                            float* g_opacity, float* g_logits, void* ws, size_t ws_bytes, cudaStream_t st) {
    sq_scene_t s;
    memset(&s, 0, sizeof(s));
    s.prims = *prims;
    s.index = *idx;
    s.grid = *grid;
    s.rays = *rays;
    s.saved = const_cast<void*>(saved);
    s.saved_bytes = saved_bytes;
    s.grad_depth = grad_depth;
    s.grad_sem = grad_sem;
    s.g_means = g_means;
    s.g_quats = g_quats;
    s.g_scales = g_scales;
    s.g_eps = g_eps;
    s.g_opacity = g_opacity;
    s.g_logits = g_logits;
    return batched_impl(SQ_OP_BWD, &s, 1, default_tuning(), ws, ws_bytes, st);
}

sq_status_t batched_api_impl(int op, const sq_scene_t* sc, int n, const sq_tuning_t* tuning, void* ws,
                             size_t ws_bytes, cudaStream_t st) {
    Tuning t = default_tuning();
    if (tuning) {
        t.fwd_lanes = tuning->fwd_lanes_per_ray;
        t.fwd_warps = tuning->fwd_warps_per_cta;
        t.bwd_warps = tuning->bwd_warps_per_cta;
        if (tuning->bwd_order != SQ_BWD_DEFAULT) t.bwd_order = tuning->bwd_order;
        t.fwd_tile = tuning->fwd_ray_tile > 0 ? tuning->fwd_ray_tile : 1;
    }
    if (t.fwd_tile < 1 || t.fwd_tile > 64) {
        set_last_error("forward ray tile %d not supported (1..64)", t.fwd_tile);
        return SQ_ERR_INVALID_ARG;
    }
    if (t.bwd_order != SQ_BWD_RAY_MAJOR && t.bwd_order != SQ_BWD_PRIMITIVE_MAJOR) {
        set_last_error("backward order %d not supported", t.bwd_order);
        return SQ_ERR_INVALID_ARG;
    }
    return batched_impl(op, sc, n, t, ws, ws_bytes, st);
}

// Times every candidate launch configuration on the given batch (forward: lanes
// per ray x warps per CTA; backward: warps per CTA) with CUDA events on the
// stream and keeps the fastest of each.  Host-synchronous.
sq_status_t autotune_impl(const sq_scene_t* sc, int n, void* ws, size_t ws_bytes, cudaStream_t st, sq_tuning_t* best,
                          float* fwd_ms, float* bwd_ms, int reps) {
    const Tuning fcand[8] = {{4, 4, 8, 0, 1},  {4, 8, 8, 0, 1},  {8, 4, 8, 0, 1},  {8, 8, 8, 0, 1},
                             {4, 4, 8, 0, 16}, {4, 8, 8, 0, 16}, {8, 4, 8, 0, 16}, {8, 8, 8, 0, 16}};
    // ray-major with 0 (the most resident warps for the batch's L), 4 or 8 warps per
    // CTA, then primitive-major
    const int bcand[4] = {0, 4, 8, 0};
    const int bord[4] = {SQ_BWD_RAY_MAJOR, SQ_BWD_RAY_MAJOR, SQ_BWD_RAY_MAJOR, SQ_BWD_PRIMITIVE_MAJOR};
    if (reps < 1) reps = 1;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_status(e, "autotune event");
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_status(e, "autotune event");
    }
    sq_status_t s = SQ_OK;
    float bestf = 1e30f, bestb = 1e30f;
    Tuning tb = default_tuning();
    for (int c = 0; c < 8 && s == SQ_OK; ++c) {
        Tuning fc = fcand[c];
        fc.bwd_order = tb.bwd_order;
        s = batched_impl(SQ_OP_FWD, sc, n, fc, ws, ws_bytes, st);  // warm-up
        if (s != SQ_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == SQ_OK; ++r) s = batched_impl(SQ_OP_FWD, sc, n, fc, ws, ws_bytes, st);
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            s = cuda_status(e, "autotune sync");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (fwd_ms) fwd_ms[c] = ms;
        if (ms < bestf) {
            bestf = ms;
            tb.fwd_lanes = fc.fwd_lanes;
            tb.fwd_warps = fc.fwd_warps;
            tb.fwd_tile = fc.fwd_tile;
        }
    }
    if (s == SQ_OK) s = batched_impl(SQ_OP_FWD, sc, n, tb, ws, ws_bytes, st);  // saved state for the backward
    bool do_bwd = s == SQ_OK;
    for (int i = 0; i < n && do_bwd; ++i) do_bwd = sc[i].saved != nullptr && sc[i].grad_depth && sc[i].grad_sem;
    for (int c = 0; c < 4 && do_bwd && s == SQ_OK; ++c) {
        Tuning t = tb;
        t.bwd_warps = bcand[c];
        t.bwd_order = bord[c];
        s = batched_impl(SQ_OP_BWD, sc, n, t, ws, ws_bytes, st);
        if (s != SQ_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == SQ_OK; ++r) s = batched_impl(SQ_OP_BWD, sc, n, t, ws, ws_bytes, st);
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            s = cuda_status(e, "autotune sync");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (bwd_ms) bwd_ms[c] = ms;
        if (ms < bestb) {
            bestb = ms;
            tb.bwd_warps = bcand[c];
            tb.bwd_order = bord[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != SQ_OK) return s;
    best->fwd_lanes_per_ray = tb.fwd_lanes;
    best->fwd_warps_per_cta = tb.fwd_warps;
    best->bwd_warps_per_cta = tb.bwd_warps;
    best->bwd_order = tb.bwd_order;
    best->fwd_ray_tile = tb.fwd_tile;
    return SQ_OK;
}

sq_status_t count_pairs_impl(const sq_index_t* idx, const sq_grid_t* grid, const sq_rays_t* rays, long long* out,
                             cudaStream_t st) {
    SceneDesc S;
    memset(&S, 0, sizeof(S));
    S.v_n = idx->v_n;
    S.g = make_grid(grid);
    S.K = rays->K;
    S.c2w = rays->cam2world;
    S.t = rays->t;
    S.n_cam = rays->n_cam;
    S.H = rays->H;
    S.W = rays->W;
    S.L = rays->L;
    S.R = (long long)rays->n_cam * rays->H * rays->W;
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(long long), st);
    if (e != cudaSuccess) return cuda_status(e, "memset count");
    if (S.R == 0) return SQ_OK;
    const long long want = (S.R * S.L + 255) / 256;
    const int blocks = (int)(want < 152LL * 16 ? want : 152LL * 16);
    SQ_LAUNCH("k_count_pairs", st, k_count_pairs<<<blocks, 256, 0, st>>>(S, reinterpret_cast<unsigned long long*>(out)));
    return SQ_OK;
}

}  // namespace sqr
