/*
 * sqr_oracle.c -- plain FP64 CPU oracle for the superquadric volume renderer
 * (SuperQuadricOcc-Render, "SQOcc-R", Sec. 3.3 of the SuperQuadricOcc paper).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or constant with the CUDA library and it is never on the product path.
 *
 * What it computes, written as the plain definitions:
 *   - Eq. 1   inside-outside function f of a superquadric in its canonical frame
 *             (absolute values under the fractional powers, Barr's form);
 *   - Eq. 2   occupancy p_o = exp(-f(x_S)), x_S = R^T (x - m), R = R(q/|q|),
 *             q = (w, x, y, z) a Hamilton local-to-world rotation;
 *   - Sec. 3.3.1  the voxel neighbourhood of every primitive and the
 *             voxel -> primitive lists (V_n counts, V_f offsets, V_sq ids sorted
 *             by id), built by walking the primitives in id order;
 *   - Eq. 4-6 per-sample alpha = min(sum p sigma, alpha_max), semantic vector
 *             s = sum p c, front-to-back weights w = T alpha, depth and semantics;
 *   - Sec. 3.3.3  the gradient of a loss through Eq. 4-6 and Eq. 1-2 to every
 *             primitive parameter (textbook chain rule, FP64);
 *   - Supp. A.4  voxelisation: density and semantic sums at voxel centres,
 *             label = argmax of the semantic sum, or "free" (= C) below tau.
 *
 * Discrete decisions (which voxel a sample falls in, a primitive's voxel
 * range) are taken exactly as the CUDA library takes them: sample positions
 * are formed in FP32 with a fixed order of IEEE operations (this file must be
 * compiled with -ffp-contract=off), voxel ranges in FP64 with a fixed order.
 * Every continuous quantity is then evaluated in FP64 from the FP32 sample
 * position.
 *
 * Parity status: every function here is pinned by tests against closed forms,
 * invariants, brute force and central finite differences; none is "parity
 * unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ----------------------------------------------------------------------- */
/* Grid and ray construction (discrete part, FP32, fixed op order)         */
/* ----------------------------------------------------------------------- */

typedef struct {
    int n[3];
    float lo[3];
    float vs[3];
    float inv_vs[3];
} ogrid_t;

static ogrid_t make_grid(const int* n, const float* lo, const float* vs) {
    ogrid_t g;
    for (int i = 0; i < 3; ++i) {
        g.n[i] = n[i];
        g.lo[i] = lo[i];
        g.vs[i] = vs[i];
        g.inv_vs[i] = 1.0f / vs[i];
    }
    return g;
}

/* Pinhole ray of pixel (u, v) through the pixel centre, OpenCV axes.
 * K = (fx, fy, cx, cy); c2w = 3x4 row-major [R | centre]. */
static void ray_of_pixel(const float* K, const float* c2w, int u, int v, float o[3], float d[3]) {
    float a = (float)u + 0.5f;
    a = a - K[2];
    float dx = a / K[0];
    float b = (float)v + 0.5f;
    b = b - K[3];
    float dy = b / K[1];
    float n2 = dx * dx + dy * dy;
    n2 = n2 + 1.0f;
    float nrm = sqrtf(n2);
    float cxn = dx / nrm, cyn = dy / nrm, czn = 1.0f / nrm;
    for (int i = 0; i < 3; ++i) {
        float di = c2w[4 * i + 0] * cxn + c2w[4 * i + 1] * cyn;
        di = di + c2w[4 * i + 2] * czn;
        d[i] = di;
        o[i] = c2w[4 * i + 3];
    }
}

/* Sample j of a ray: x = o + t d (FP32), voxel id (z fastest) or -1 if outside. */
static long long sample_voxel(const ogrid_t* g, const float o[3], const float d[3], float t, float x[3]) {
    int idx[3];
    int inside = 1;
    for (int i = 0; i < 3; ++i) {
        float td = t * d[i];
        x[i] = o[i] + td;
        float u = (x[i] - g->lo[i]) * g->inv_vs[i];
        if (!(u >= 0.0f && u < (float)g->n[i])) {
            inside = 0;
            idx[i] = 0;
        } else {
            idx[i] = (int)floorf(u);
        }
    }
    if (!inside) return -1;
    return ((long long)idx[0] * g->n[1] + idx[1]) * g->n[2] + idx[2];
}

/* ----------------------------------------------------------------------- */
/* Primitive geometry (FP64)                                               */
/* ----------------------------------------------------------------------- */

typedef struct {
    double m[3];
    double q[4];   /* raw quaternion */
    double qn[4];  /* normalised */
    double qnorm;
    double R[9];   /* local -> world, row-major */
    double s[3];
    double e1, e2;
    double sigma;
    const double* c; /* C class values (FP64) */
} oprim_t;

/* Normalise q and form the Hamilton rotation matrix (local -> world). */
static void quat_rotation(const double q[4], double qn[4], double* qnorm, double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double nq = sqrt(((w * w + x * x) + y * y) + z * z);
    w = w / nq; x = x / nq; y = y / nq; z = z / nq;
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    *qnorm = nq;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static oprim_t load_prim(int k, int C, const float* means, const float* quats, const float* scales,
                         const float* eps, const float* opacity, const double* logits) {
    oprim_t p;
    for (int i = 0; i < 3; ++i) { p.m[i] = means[3 * k + i]; p.s[i] = scales[3 * k + i]; }
    for (int i = 0; i < 4; ++i) p.q[i] = quats[4 * k + i];
    quat_rotation(p.q, p.qn, &p.qnorm, p.R);
    p.e1 = eps[2 * k + 0];
    p.e2 = eps[2 * k + 1];
    p.sigma = opacity[k];
    p.c = logits + (size_t)k * C;
    return p;
}

/* Canonical-frame coordinates x_S = R^T (x - m). */
static void to_local(const oprim_t* p, const double x[3], double d[3], double xl[3]) {
    for (int i = 0; i < 3; ++i) d[i] = x[i] - p->m[i];
    for (int j = 0; j < 3; ++j) xl[j] = p->R[0 * 3 + j] * d[0] + p->R[1 * 3 + j] * d[1] + p->R[2 * 3 + j] * d[2];
}

/* Eq. 1: f = ((|x|/sx)^(2/e2) + (|y|/sy)^(2/e2))^(e2/e1) + (|z|/sz)^(2/e1). */
double orc_sq_f(const double* xl, const double* s, double e1, double e2) {
    double a = fabs(xl[0]) / s[0], b = fabs(xl[1]) / s[1], c = fabs(xl[2]) / s[2];
    double A = pow(a, 2.0 / e2) + pow(b, 2.0 / e2);
    return pow(A, e2 / e1) + pow(c, 2.0 / e1);
}

/* Eq. 2: p_o(x) = exp(-f(R^T (x - m))). */
double orc_sq_p(const double* x, const double* m, const double* q, const double* s, double e1, double e2) {
    oprim_t p;
    for (int i = 0; i < 3; ++i) { p.m[i] = m[i]; p.s[i] = s[i]; }
    for (int i = 0; i < 4; ++i) p.q[i] = q[i];
    quat_rotation(p.q, p.qn, &p.qnorm, p.R);
    double d[3], xl[3];
    to_local(&p, x, d, xl);
    return exp(-orc_sq_f(xl, p.s, e1, e2));
}

/* Gradient of f with respect to the primitive's raw parameters, at world point x.
 * Outputs: df/dm (3), df/dq (4, raw quaternion), df/ds (3), df/d(e1,e2) (2).
 * Returns f.  Terms whose base is exactly zero contribute 0 (their limit). */
static double sq_f_grad(const oprim_t* p, const double x[3], double gm[3], double gq[4], double gs[3], double ge[2]) {
    double d[3], xl[3];
    to_local(p, x, d, xl);
    const double e1 = p->e1, e2 = p->e2;
    const double ea = 2.0 / e2, eb = e2 / e1, ec = 2.0 / e1;
    double a = fabs(xl[0]) / p->s[0], b = fabs(xl[1]) / p->s[1], c = fabs(xl[2]) / p->s[2];
    double pa = pow(a, ea), pb = pow(b, ea), pc = pow(c, ec);
    double A = pa + pb;
    double Aeb = pow(A, eb);
    double f = Aeb + pc;

    /* df/da = eb A^(eb-1) * ea a^(ea-1); df/dc = ec c^(ec-1) */
    double dfa = (a > 0.0 && A > 0.0) ? eb * pow(A, eb - 1.0) * ea * pow(a, ea - 1.0) : 0.0;
    double dfb = (b > 0.0 && A > 0.0) ? eb * pow(A, eb - 1.0) * ea * pow(b, ea - 1.0) : 0.0;
    double dfc = (c > 0.0) ? ec * pow(c, ec - 1.0) : 0.0;

    double sgn[3];
    for (int i = 0; i < 3; ++i) sgn[i] = (xl[i] > 0.0) ? 1.0 : ((xl[i] < 0.0) ? -1.0 : 0.0);
    double gxl[3] = {dfa * sgn[0] / p->s[0], dfb * sgn[1] / p->s[1], dfc * sgn[2] / p->s[2]};

    /* a = |x|/sx  =>  da/dsx = -a/sx */
    gs[0] = -dfa * a / p->s[0];
    gs[1] = -dfb * b / p->s[1];
    gs[2] = -dfc * c / p->s[2];

    /* exponents: ea = 2/e2, eb = e2/e1, ec = 2/e1 */
    double lnA = (A > 0.0) ? log(A) : 0.0;
    double dA_dea = ((pa > 0.0) ? pa * log(a) : 0.0) + ((pb > 0.0) ? pb * log(b) : 0.0);
    double dAeb_de2 = (A > 0.0) ? Aeb * (lnA * (1.0 / e1) + eb * (dA_dea / A) * (-2.0 / (e2 * e2))) : 0.0;
    double dAeb_de1 = (A > 0.0) ? Aeb * lnA * (-e2 / (e1 * e1)) : 0.0;
    double dpc_de1 = (pc > 0.0) ? pc * log(c) * (-2.0 / (e1 * e1)) : 0.0;
    ge[0] = dAeb_de1 + dpc_de1;
    ge[1] = dAeb_de2;

    /* x_S = R^T (x - m): df/dm = -R gxl, df/dR_ij = d_i gxl_j */
    for (int i = 0; i < 3; ++i) gm[i] = -(p->R[3 * i + 0] * gxl[0] + p->R[3 * i + 1] * gxl[1] + p->R[3 * i + 2] * gxl[2]);
    double gR[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gR[3 * i + j] = d[i] * gxl[j];

    /* dR/dq for the normalised quaternion (w, x, y, z) */
    const double w = p->qn[0], x_ = p->qn[1], y = p->qn[2], z = p->qn[3];
    double gqn[4];
    gqn[0] = gR[1] * (-2 * z) + gR[2] * (2 * y) + gR[3] * (2 * z) + gR[5] * (-2 * x_) + gR[6] * (-2 * y) + gR[7] * (2 * x_);
    gqn[1] = gR[1] * (2 * y) + gR[2] * (2 * z) + gR[3] * (2 * y) + gR[4] * (-4 * x_) + gR[5] * (-2 * w) + gR[6] * (2 * z) +
             gR[7] * (2 * w) + gR[8] * (-4 * x_);
    gqn[2] = gR[0] * (-4 * y) + gR[1] * (2 * x_) + gR[2] * (2 * w) + gR[3] * (2 * x_) + gR[5] * (2 * z) + gR[6] * (-2 * w) +
             gR[7] * (2 * z) + gR[8] * (-4 * y);
    gqn[3] = gR[0] * (-4 * z) + gR[1] * (-2 * w) + gR[2] * (2 * x_) + gR[3] * (2 * w) + gR[4] * (-4 * z) + gR[5] * (2 * y) +
             gR[6] * (2 * x_) + gR[7] * (2 * y);
    /* through q_n = q / |q|:  dq = (gqn - qn (qn . gqn)) / |q| */
    double dot = gqn[0] * w + gqn[1] * x_ + gqn[2] * y + gqn[3] * z;
    for (int i = 0; i < 4; ++i) gq[i] = (gqn[i] - p->qn[i] * dot) / p->qnorm;
    return f;
}

/* ----------------------------------------------------------------------- */
/* Voxel neighbourhoods and the voxel -> primitive index (Sec. 3.3.1)       */
/* ----------------------------------------------------------------------- */

static int near_integer(double u) { return fabs(u - floor(u + 0.5)) < 1e-9; }

/* Per primitive, an inclusive voxel box [i0,i1]x[j0,j1]x[k0,k1] clipped to the grid,
 * written as ranges[6k..6k+5] = (i0, i1, j0, j1, k0, k1); empty boxes are
 * (0,-1,0,-1,0,-1).
 *   mode 0 (OBB): the level set p_o >= tau_cut of a superquadric is contained in
 *     its local box |x_i| <= s_i * Kc^(e1/2), Kc = ln(1/tau_cut) (along a local
 *     axis f = (|x_i|/s_i)^(2/e1), and every other coordinate only adds to f);
 *     the world AABB of that oriented box has half-width sum_i |R_ji| h_i.
 *   mode 1 (cube): the voxel containing the centre +- nv voxels (the paper's
 *     cubic neighbourhood N_v).
 *   mode 2 (opacity-aware OBB, the index refinement the paper names as future
 *     work): as mode 0 for the level set sigma_k p_o >= tau_cut, i.e.
 *     Kc_k = ln(sigma_k) - ln(tau_cut); a primitive with sigma_k <= tau_cut has
 *     no voxels.
 * Returns the number of primitives whose box bounds fall within 1e-9 of a
 * voxel boundary (where a one-ulp difference could move the box). */
long long orc_ranges(int n, const float* means, const float* quats, const float* scales, const float* eps,
                     const float* opacity, const int* gn, const float* glo, const float* gvs, int mode,
                     float tau_cut, int nv, int* ranges) {
    long long ties = 0;
    const double log_kc0 = log(-log((double)tau_cut));
    for (int k = 0; k < n; ++k) {
        double q[4], qn[4], qnorm, R[9];
        for (int i = 0; i < 4; ++i) q[i] = quats[4 * k + i];
        quat_rotation(q, qn, &qnorm, R);
        double e1 = eps[2 * k + 0];
        double log_kc = log_kc0;
        if (mode == 2) {
            if (!((double)opacity[k] > (double)tau_cut)) {
                for (int j = 0; j < 3; ++j) {
                    ranges[6 * k + 2 * j + 0] = 0;
                    ranges[6 * k + 2 * j + 1] = -1;
                }
                continue;
            }
            log_kc = log(log((double)opacity[k]) - log((double)tau_cut));
        }
        double ext = exp((0.5 * e1) * log_kc);
        double h[3];
        for (int i = 0; i < 3; ++i) h[i] = (double)scales[3 * k + i] * ext;
        int lo_i[3], hi_i[3], empty = 0, tie = 0;
        for (int j = 0; j < 3; ++j) {
            double m = means[3 * k + j];
            double lo = glo[j], vs = gvs[j];
            double ulo, uhi;
            if (mode != 1) {
                double hw = fabs(R[3 * j + 0]) * h[0] + fabs(R[3 * j + 1]) * h[1];
                hw = hw + fabs(R[3 * j + 2]) * h[2];
                ulo = ((m - hw) - lo) / vs;
                uhi = ((m + hw) - lo) / vs;
                if (near_integer(ulo) && ulo > -1.0 && ulo < gn[j] + 1.0) tie = 1;
                if (near_integer(uhi) && uhi > -1.0 && uhi < gn[j] + 1.0) tie = 1;
            } else {
                double uc = (m - lo) / vs;
                if (near_integer(uc) && uc > -1.0 - nv && uc < gn[j] + 1.0 + nv) tie = 1;
                double cf = floor(fmin(fmax(uc, -1.0 - nv), (double)gn[j] + nv));
                ulo = cf - nv;
                uhi = cf + nv;
            }
            if (!(ulo == ulo) || !(uhi == uhi)) { empty = 1; continue; }
            double a = floor(fmin(fmax(ulo, -1.0), (double)gn[j]));
            double b = floor(fmin(fmax(uhi, -1.0), (double)gn[j]));
            int i0 = (int)a, i1 = (int)b;
            if (i0 < 0) i0 = 0;
            if (i1 > gn[j] - 1) i1 = gn[j] - 1;
            if (i0 > i1) empty = 1;
            lo_i[j] = i0;
            hi_i[j] = i1;
        }
        ties += tie;
        for (int j = 0; j < 3; ++j) {
            ranges[6 * k + 2 * j + 0] = empty ? 0 : lo_i[j];
            ranges[6 * k + 2 * j + 1] = empty ? -1 : hi_i[j];
        }
    }
    return ties;
}

/* Voxel -> primitive lists.  v_n[v] = number of primitives whose box holds v,
 * v_f = exclusive prefix sum of v_n, v_sq[v_f[v] .. v_f[v]+v_n[v]) = those
 * primitive ids ascending (ids are appended while walking k = 0..n-1).
 * Voxel id = (ix*ny + iy)*nz + iz.  Returns P = total entries; v_sq is only
 * written when P <= cap. */
long long orc_index(int n, const int* ranges, const int* gn, int* v_n, int* v_f, int* v_sq, long long cap) {
    const long long nvox = (long long)gn[0] * gn[1] * gn[2];
    memset(v_n, 0, sizeof(int) * nvox);
    for (int k = 0; k < n; ++k) {
        const int* r = ranges + 6 * k;
        for (int ix = r[0]; ix <= r[1]; ++ix)
            for (int iy = r[2]; iy <= r[3]; ++iy)
                for (int iz = r[4]; iz <= r[5]; ++iz) v_n[((long long)ix * gn[1] + iy) * gn[2] + iz] += 1;
    }
    long long P = 0;
    for (long long v = 0; v < nvox; ++v) { v_f[v] = (int)P; P += v_n[v]; }
    if (P > cap || v_sq == NULL) return P;
    int* fill = (int*)calloc((size_t)nvox, sizeof(int));
    for (int k = 0; k < n; ++k) {
        const int* r = ranges + 6 * k;
        for (int ix = r[0]; ix <= r[1]; ++ix)
            for (int iy = r[2]; iy <= r[3]; ++iy)
                for (int iz = r[4]; iz <= r[5]; ++iz) {
                    long long v = ((long long)ix * gn[1] + iy) * gn[2] + iz;
                    v_sq[v_f[v] + fill[v]] = k;
                    fill[v] += 1;
                }
    }
    free(fill);
    return P;
}

/* ----------------------------------------------------------------------- */
/* Forward (Eq. 4-6) and backward (Sec. 3.3.3)                              */
/* ----------------------------------------------------------------------- */

typedef struct {
    int n, C;
    const float *means, *quats, *scales, *eps, *opacity;
    const double* logits;
    ogrid_t g;
    const int *v_n, *v_f, *v_sq;
    int n_cam, H, W, L;
    const float *K, *c2w, *t;
    double kappa, alpha_max;
} oscene_t;

static oscene_t make_scene(int n, int C, const float* means, const float* quats, const float* scales,
                           const float* eps, const float* opacity, const double* logits, const int* gn,
                           const float* glo, const float* gvs, const int* v_n, const int* v_f, const int* v_sq,
                           int n_cam, int H, int W, const float* K, const float* c2w, int L, const float* t,
                           double kappa, double alpha_max) {
    oscene_t s;
    s.n = n; s.C = C;
    s.means = means; s.quats = quats; s.scales = scales; s.eps = eps; s.opacity = opacity; s.logits = logits;
    s.g = make_grid(gn, glo, gvs);
    s.v_n = v_n; s.v_f = v_f; s.v_sq = v_sq;
    s.n_cam = n_cam; s.H = H; s.W = W; s.L = L;
    s.K = K; s.c2w = c2w; s.t = t;
    s.kappa = kappa; s.alpha_max = alpha_max;
    return s;
}

static void ray_of_id(const oscene_t* s, long long r, float o[3], float d[3]) {
    long long hw = (long long)s->H * s->W;
    int cam = (int)(r / hw);
    long long pix = r - (long long)cam * hw;
    int v = (int)(pix / s->W), u = (int)(pix - (long long)v * s->W);
    ray_of_pixel(s->K + 4 * cam, s->c2w + 12 * cam, u, v, o, d);
}

/* Per-sample quantities of one ray: alpha (clamped), raw sum, semantic vector,
 * transmittance before the sample.  Returns the number of samples composited
 * (L, or fewer when early termination with kappa > 0 stopped the ray). */
typedef struct {
    double* alpha;   /* [L] */
    double* ssum;    /* [L] raw sum of p*sigma */
    double* sem;     /* [L*C] */
    double* T;       /* [L+1] */
    long long* vox;  /* [L] */
} otrace_t;

static int trace_ray(const oscene_t* s, long long r, otrace_t* tr) {
    float o[3], d[3];
    ray_of_id(s, r, o, d);
    const int C = s->C;
    double T = 1.0;
    int used = 0;
    for (int j = 0; j < s->L; ++j) {
        float xf[3];
        long long v = sample_voxel(&s->g, o, d, s->t[j], xf);
        double x[3] = {xf[0], xf[1], xf[2]};
        double sum = 0.0;
        double* sem = tr->sem + (size_t)j * C;
        for (int c = 0; c < C; ++c) sem[c] = 0.0;
        tr->vox[j] = v;
        if (v >= 0) {
            int beg = s->v_f[v], cnt = s->v_n[v];
            for (int e = 0; e < cnt; ++e) {
                int k = s->v_sq[beg + e];
                oprim_t p = load_prim(k, C, s->means, s->quats, s->scales, s->eps, s->opacity, s->logits);
                double dd[3], xl[3];
                to_local(&p, x, dd, xl);
                double po = exp(-orc_sq_f(xl, p.s, p.e1, p.e2));
                sum += po * p.sigma;
                for (int c = 0; c < C; ++c) sem[c] += po * (double)p.c[c];
            }
        }
        double alpha = sum < s->alpha_max ? sum : s->alpha_max;
        tr->alpha[j] = alpha;
        tr->ssum[j] = sum;
        tr->T[j] = T;
        T = T * (1.0 - alpha);
        used = j + 1;
        if (s->kappa > 0.0 && T < s->kappa) break;
    }
    tr->T[used] = T;
    return used;
}

static otrace_t alloc_trace(int L, int C) {
    otrace_t tr;
    tr.alpha = (double*)malloc(sizeof(double) * L);
    tr.ssum = (double*)malloc(sizeof(double) * L);
    tr.sem = (double*)malloc(sizeof(double) * (size_t)L * C);
    tr.T = (double*)malloc(sizeof(double) * (L + 1));
    tr.vox = (long long*)malloc(sizeof(long long) * L);
    return tr;
}

static void free_trace(otrace_t* tr) {
    free(tr->alpha); free(tr->ssum); free(tr->sem); free(tr->T); free(tr->vox);
}

static int set_threads(int n_threads) {
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
    return nt;
#else
    (void)n_threads;
    return 1;
#endif
}

/* Forward render of the rays listed in ray_ids (or all rays when ray_ids is
 * NULL).  Outputs per listed ray: depth = sum_j w_j t_j, sem[C] = sum_j w_j s_j,
 * t_final = transmittance after the last composited sample, n_used = samples
 * composited. */
int orc_render_fwd(int n, int C, const float* means, const float* quats, const float* scales, const float* eps,
                   const float* opacity, const double* logits, const int* gn, const float* glo, const float* gvs,
                   const int* v_n, const int* v_f, const int* v_sq, int n_cam, int H, int W, const float* K,
                   const float* c2w, int L, const float* t, double kappa, double alpha_max, const long long* ray_ids,
                   long long n_rays, double* depth, double* sem, double* t_final, int* n_used, int n_threads) {
    oscene_t s = make_scene(n, C, means, quats, scales, eps, opacity, logits, gn, glo, gvs, v_n, v_f, v_sq, n_cam, H,
                            W, K, c2w, L, t, kappa, alpha_max);
    long long total = ray_ids ? n_rays : (long long)n_cam * H * W;
    int nt = set_threads(n_threads);
#pragma omp parallel num_threads(nt)
    {
        otrace_t tr = alloc_trace(L, C);
#pragma omp for schedule(dynamic, 64)
        for (long long i = 0; i < total; ++i) {
            long long r = ray_ids ? ray_ids[i] : i;
            int used = trace_ray(&s, r, &tr);
            double D = 0.0;
            double* S = sem + (size_t)i * C;
            for (int c = 0; c < C; ++c) S[c] = 0.0;
            for (int j = 0; j < used; ++j) {
                double w = tr.T[j] * tr.alpha[j];
                D += w * (double)t[j];
                for (int c = 0; c < C; ++c) S[c] += w * tr.sem[(size_t)j * C + c];
            }
            depth[i] = D;
            if (t_final) t_final[i] = tr.T[used];
            if (n_used) n_used[i] = used;
        }
        free_trace(&tr);
    }
    return 0;
}

/* Per-sample trace of one ray for tests: alpha, raw sum, T before each sample,
 * voxel id.  Returns samples composited. */
int orc_trace_ray(int n, int C, const float* means, const float* quats, const float* scales, const float* eps,
                  const float* opacity, const double* logits, const int* gn, const float* glo, const float* gvs,
                  const int* v_n, const int* v_f, const int* v_sq, int n_cam, int H, int W, const float* K,
                  const float* c2w, int L, const float* t, double kappa, double alpha_max, long long ray,
                  double* alpha, double* ssum, double* T, long long* vox, float* xyz) {
    oscene_t s = make_scene(n, C, means, quats, scales, eps, opacity, logits, gn, glo, gvs, v_n, v_f, v_sq, n_cam, H,
                            W, K, c2w, L, t, kappa, alpha_max);
    otrace_t tr = alloc_trace(L, C);
    int used = trace_ray(&s, ray, &tr);
    for (int j = 0; j < L; ++j) {
        alpha[j] = j < used ? tr.alpha[j] : 0.0;
        ssum[j] = j < used ? tr.ssum[j] : 0.0;
        vox[j] = j < used ? tr.vox[j] : -1;
    }
    for (int j = 0; j <= used; ++j) T[j] = tr.T[j];
    for (int j = used + 1; j <= L; ++j) T[j] = tr.T[used];
    if (xyz) {
        float o[3], d[3];
        ray_of_id(&s, ray, o, d);
        for (int j = 0; j < L; ++j) {
            float xf[3];
            sample_voxel(&s.g, o, d, t[j], xf);
            for (int i = 0; i < 3; ++i) xyz[3 * j + i] = xf[i];
        }
    }
    free_trace(&tr);
    return used;
}

/* Backward: given cotangents gD = dL/dD (per listed ray) and gS = dL/dS [C],
 * accumulate dL/d(params) over the listed rays.  Per ray:
 *   v_j = gD t_j + <gS, s_j>
 *   dL/dalpha_j = T_j (v_j - U_j),  U_j = sum_{i>j} alpha_i v_i prod_{j<l<i} (1 - alpha_l)
 *   (zero where the clamp alpha = alpha_max is active, i.e. raw sum > alpha_max)
 *   per pair (j, k):  dL/dsigma_k += G_j p,  dL/dc_k += w_j p gS,
 *                     dL/dp = G_j sigma_k + w_j <gS, c_k>,  dL/df = -p dL/dp,
 *                     and df/d(m, q, s, e) from sq_f_grad.
 * Gradient outputs are overwritten (not accumulated into). */
int orc_render_bwd(int n, int C, const float* means, const float* quats, const float* scales, const float* eps,
                   const float* opacity, const double* logits, const int* gn, const float* glo, const float* gvs,
                   const int* v_n, const int* v_f, const int* v_sq, int n_cam, int H, int W, const float* K,
                   const float* c2w, int L, const float* t, double kappa, double alpha_max, const long long* ray_ids,
                   long long n_rays, const double* grad_depth, const double* grad_sem, double* g_means,
                   double* g_quats, double* g_scales, double* g_eps, double* g_opacity, double* g_logits,
                   int n_threads) {
    oscene_t s = make_scene(n, C, means, quats, scales, eps, opacity, logits, gn, glo, gvs, v_n, v_f, v_sq, n_cam, H,
                            W, K, c2w, L, t, kappa, alpha_max);
    long long total = ray_ids ? n_rays : (long long)n_cam * H * W;
    const int NP = 13 + C; /* m3 q4 s3 e2 sigma1 c[C] */
    int nt = set_threads(n_threads);
    double* acc = (double*)calloc((size_t)nt * n * NP, sizeof(double));
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* G = acc + (size_t)tid * n * NP;
        otrace_t tr = alloc_trace(L, C);
        double* v = (double*)malloc(sizeof(double) * L);
        double* dA = (double*)malloc(sizeof(double) * L);
#pragma omp for schedule(dynamic, 64)
        for (long long i = 0; i < total; ++i) {
            long long r = ray_ids ? ray_ids[i] : i;
            float o[3], d[3];
            ray_of_id(&s, r, o, d);
            int used = trace_ray(&s, r, &tr);
            const double gD = grad_depth[i];
            const double* gS = grad_sem + (size_t)i * C;
            for (int j = 0; j < used; ++j) {
                double vj = gD * (double)t[j];
                for (int c = 0; c < C; ++c) vj += gS[c] * tr.sem[(size_t)j * C + c];
                v[j] = vj;
            }
            double U = 0.0;
            for (int j = used - 1; j >= 0; --j) {
                double g = tr.T[j] * (v[j] - U);
                dA[j] = (tr.ssum[j] > s.alpha_max) ? 0.0 : g;
                U = tr.alpha[j] * v[j] + (1.0 - tr.alpha[j]) * U;
            }
            for (int j = 0; j < used; ++j) {
                long long vx = tr.vox[j];
                if (vx < 0) continue;
                float xf[3];
                sample_voxel(&s.g, o, d, t[j], xf);
                double x[3] = {xf[0], xf[1], xf[2]};
                double w = tr.T[j] * tr.alpha[j];
                int beg = s.v_f[vx], cnt = s.v_n[vx];
                for (int e = 0; e < cnt; ++e) {
                    int k = s.v_sq[beg + e];
                    oprim_t p = load_prim(k, C, means, quats, scales, eps, opacity, logits);
                    double gm[3], gq[4], gs[3], ge[2];
                    double f = sq_f_grad(&p, x, gm, gq, gs, ge);
                    double po = exp(-f);
                    double cdot = 0.0;
                    for (int c = 0; c < C; ++c) cdot += gS[c] * (double)p.c[c];
                    double gp = dA[j] * p.sigma + w * cdot;
                    double gf = -po * gp;
                    double* Gk = G + (size_t)k * NP;
                    for (int a = 0; a < 3; ++a) Gk[a] += gf * gm[a];
                    for (int a = 0; a < 4; ++a) Gk[3 + a] += gf * gq[a];
                    for (int a = 0; a < 3; ++a) Gk[7 + a] += gf * gs[a];
                    for (int a = 0; a < 2; ++a) Gk[10 + a] += gf * ge[a];
                    Gk[12] += dA[j] * po;
                    for (int c = 0; c < C; ++c) Gk[13 + c] += w * po * gS[c];
                }
            }
        }
        free(v);
        free(dA);
        free_trace(&tr);
    }
    for (int k = 0; k < n; ++k) {
        double sum[64 + 13];
        double* tot = NP <= 77 ? sum : (double*)malloc(sizeof(double) * NP);
        for (int a = 0; a < NP; ++a) tot[a] = 0.0;
        for (int th = 0; th < nt; ++th)
            for (int a = 0; a < NP; ++a) tot[a] += acc[((size_t)th * n + k) * NP + a];
        for (int a = 0; a < 3; ++a) g_means[3 * k + a] = tot[a];
        for (int a = 0; a < 4; ++a) g_quats[4 * k + a] = tot[3 + a];
        for (int a = 0; a < 3; ++a) g_scales[3 * k + a] = tot[7 + a];
        for (int a = 0; a < 2; ++a) g_eps[2 * k + a] = tot[10 + a];
        g_opacity[k] = tot[12];
        for (int c = 0; c < C; ++c) g_logits[(size_t)k * C + c] = tot[13 + c];
        if (tot != sum) free(tot);
    }
    free(acc);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Voxelisation (Supp. A.4)                                                 */
/* ----------------------------------------------------------------------- */

/* At each listed voxel centre p (FP32: lo + (i + 0.5) vs, then promoted):
 * density = sum_{k in Q(v)} p_o sigma_k, sem[C] = sum p_o c_k,
 * label = argmax_c sem (lowest index on ties) if density >= tau, else C.
 * voxel_ids NULL means every voxel in id order. */
int orc_query_grid(int n, int C, const float* means, const float* quats, const float* scales, const float* eps,
                   const float* opacity, const double* logits, const int* gn, const float* glo, const float* gvs,
                   const int* v_n, const int* v_f, const int* v_sq, double tau, const long long* voxel_ids,
                   long long n_sel, double* density, double* sem, int* label, int n_threads) {
    ogrid_t g = make_grid(gn, glo, gvs);
    long long nvox = (long long)gn[0] * gn[1] * gn[2];
    long long total = voxel_ids ? n_sel : nvox;
    int nt = set_threads(n_threads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 256)
    for (long long i = 0; i < total; ++i) {
        long long v = voxel_ids ? voxel_ids[i] : i;
        int iz = (int)(v % gn[2]);
        int iy = (int)((v / gn[2]) % gn[1]);
        int ix = (int)(v / ((long long)gn[1] * gn[2]));
        int id[3] = {ix, iy, iz};
        double x[3];
        for (int a = 0; a < 3; ++a) {
            float c = (float)id[a] + 0.5f;
            float cv = c * g.vs[a];
            float xf = g.lo[a] + cv;
            x[a] = xf;
        }
        double dens = 0.0;
        double* S = sem + (size_t)i * C;
        for (int c = 0; c < C; ++c) S[c] = 0.0;
        int beg = v_f[v], cnt = v_n[v];
        for (int e = 0; e < cnt; ++e) {
            int k = v_sq[beg + e];
            oprim_t p = load_prim(k, C, means, quats, scales, eps, opacity, logits);
            double dd[3], xl[3];
            to_local(&p, x, dd, xl);
            double po = exp(-orc_sq_f(xl, p.s, p.e1, p.e2));
            dens += po * p.sigma;
            for (int c = 0; c < C; ++c) S[c] += po * (double)p.c[c];
        }
        density[i] = dens;
        if (label) {
            int best = 0;
            for (int c = 1; c < C; ++c)
                if (S[c] > S[best]) best = c;
            label[i] = dens >= tau ? best : C;
        }
    }
    return 0;
}

/* Gradient of sum_v gd[v] density[v] + sum_{v,c} gs[v,c] sem[v,c] over the listed
 * voxels (voxel_ids NULL: every voxel; gd, gs indexed by position in that list)
 * with respect to every primitive parameter, the index held fixed.  Per pair
 * (voxel v, k in Q(v)): dL/dp_o = gd sigma_k + <gs, c_k>, so
 * dL/dtheta += -p_o dL/dp_o df/dtheta, dL/dsigma_k += gd p_o and
 * dL/dc_k += gs p_o.  Serial, outputs overwritten. */
int orc_query_grid_bwd(int n, int C, const float* means, const float* quats, const float* scales, const float* eps,
                       const float* opacity, const double* logits, const int* gn, const float* glo, const float* gvs,
                       const int* v_n, const int* v_f, const int* v_sq, const long long* voxel_ids, long long n_sel,
                       const double* gd, const double* gs, double* g_means, double* g_quats, double* g_scales,
                       double* g_eps, double* g_opacity, double* g_logits) {
    ogrid_t g = make_grid(gn, glo, gvs);
    long long nvox = (long long)gn[0] * gn[1] * gn[2];
    long long total = voxel_ids ? n_sel : nvox;
    memset(g_means, 0, sizeof(double) * 3 * n);
    memset(g_quats, 0, sizeof(double) * 4 * n);
    memset(g_scales, 0, sizeof(double) * 3 * n);
    memset(g_eps, 0, sizeof(double) * 2 * n);
    memset(g_opacity, 0, sizeof(double) * n);
    memset(g_logits, 0, sizeof(double) * (size_t)n * C);
    for (long long i = 0; i < total; ++i) {
        long long v = voxel_ids ? voxel_ids[i] : i;
        int iz = (int)(v % gn[2]);
        int iy = (int)((v / gn[2]) % gn[1]);
        int ix = (int)(v / ((long long)gn[1] * gn[2]));
        int id[3] = {ix, iy, iz};
        double x[3];
        for (int a = 0; a < 3; ++a) {
            float c = (float)id[a] + 0.5f;
            float cv = c * g.vs[a];
            float xf = g.lo[a] + cv;
            x[a] = xf;
        }
        const double* GS = gs + (size_t)i * C;
        int beg = v_f[v], cnt = v_n[v];
        for (int e = 0; e < cnt; ++e) {
            int k = v_sq[beg + e];
            oprim_t p = load_prim(k, C, means, quats, scales, eps, opacity, logits);
            double gm[3], gq[4], gsc[3], ge[2];
            double f = sq_f_grad(&p, x, gm, gq, gsc, ge);
            double po = exp(-f);
            double cd = 0.0;
            for (int c = 0; c < C; ++c) cd += GS[c] * (double)p.c[c];
            double gf = -po * (gd[i] * p.sigma + cd);
            for (int a = 0; a < 3; ++a) g_means[3 * k + a] += gf * gm[a];
            for (int a = 0; a < 4; ++a) g_quats[4 * k + a] += gf * gq[a];
            for (int a = 0; a < 3; ++a) g_scales[3 * k + a] += gf * gsc[a];
            for (int a = 0; a < 2; ++a) g_eps[2 * k + a] += gf * ge[a];
            g_opacity[k] += gd[i] * po;
            for (int c = 0; c < C; ++c) g_logits[(size_t)k * C + c] += GS[c] * po;
        }
    }
    return 0;
}

/* FP32 sample positions and voxel ids of one ray (the discrete rule alone). */
void orc_ray_samples(const float* K, const float* c2w, int u, int v, int L, const float* t, const int* gn,
                     const float* glo, const float* gvs, float* xyz, long long* vox) {
    ogrid_t g = make_grid(gn, glo, gvs);
    float o[3], d[3];
    ray_of_pixel(K, c2w, u, v, o, d);
    for (int j = 0; j < L; ++j) vox[j] = sample_voxel(&g, o, d, t[j], xyz + 3 * j);
}

/* Voxel id (-1 outside the grid) of sample j of ray r at vox[r * L + j], for
 * every ray of the rig (Sec. 3.3.1: the sample x = o + t_j d and the voxel
 * floor((x - lo) / vs), by the FP32 rule of sample_voxel). */
void orc_sample_voxels(int n_cam, int H, int W, const float* K, const float* c2w, int L, const float* t,
                       const int* gn, const float* glo, const float* gvs, int* vox, int n_threads) {
    ogrid_t g = make_grid(gn, glo, gvs);
    long long R = (long long)n_cam * H * W;
    int nt = set_threads(n_threads);
#pragma omp parallel for num_threads(nt) schedule(static)
    for (long long r = 0; r < R; ++r) {
        int cam = (int)(r / ((long long)H * W));
        long long pix = r - (long long)cam * H * W;
        int v = (int)(pix / W), u = (int)(pix - (long long)v * W);
        float o[3], d[3], x[3];
        ray_of_pixel(K + 4 * cam, c2w + 12 * cam, u, v, o, d);
        for (int j = 0; j < L; ++j) vox[r * L + j] = (int)sample_voxel(&g, o, d, t[j], x);
    }
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
