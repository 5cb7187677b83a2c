/*
 * sqr.h -- C ABI of the GB300 superquadric volume renderer (SuperQuadricOcc-Render).
 *
 * The renderer of the SuperQuadricOcc paper (Sec. 3.3): a scene of N
 * superquadrics S_i = {m_i, s_i, r_i, eps_i, sigma_i, c_i} (Sec. 3.1) is
 * rendered by marching L samples along every pixel ray; each sample only
 * queries the superquadrics listed in its voxel (Sec. 3.3.1), sums their
 * occupancy p_o = exp(-f(x_S)) (Eq. 1-2) into an alpha and a semantic vector
 * (Eq. 4), and is alpha-composited front to back into a depth and a semantic
 * map (Eq. 5-6).  The backward pass (Sec. 3.3.3) returns the gradient of a
 * loss with respect to every superquadric parameter.  The voxelisation query
 * (Supp. A.4) evaluates density and semantics at voxel centres.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers to contiguous, row-major FP32 (or
 *    int32 / int64 where stated) memory owned by the caller.  The library
 *    never allocates device memory; scratch comes from the caller's workspace
 *    (size from sq_workspace_size, 256-byte aligned pointer).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream and never synchronise the host.
 *  - Argument errors are detected on the host before any launch and return
 *    SQ_ERR_INVALID_ARG; launch failures return SQ_ERR_CUDA.  Data-dependent
 *    errors (index capacity overflow, parameters outside their domain) are
 *    written to the device status word sq_index_t.status, read by the caller
 *    after the stream completes.
 *  - Quaternions are (w, x, y, z), a Hamilton local-to-world rotation; the
 *    canonical-frame point is x_S = R(q/|q|)^T (x - m) (Eq. 2).
 *  - Cameras are OpenCV pinholes: K[cam] = (fx, fy, cx, cy); cam2world[cam] is
 *    3x4 row-major [R | centre].  Ray r = (cam*H + v)*W + u goes through the
 *    centre of pixel (u, v).  Sample j sits at x = o + t[j] d.
 *  - The voxel of a point is floor((x - lo) * (1/vs)) per axis (FP32, fixed
 *    op order); voxel id = (ix*ny + iy)*nz + iz.  Samples outside the grid
 *    contribute alpha = 0 and s = 0 (they are skipped, Sec. 3.3.2).
 */
#ifndef SQR_H
#define SQR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SQ_OK = 0,
    SQ_ERR_INVALID_ARG = 1, /* bad size, null pointer, out-of-domain option */
    SQ_ERR_CAPACITY = 2,    /* index entries exceed sq_index_t.capacity (device status only) */
    SQ_ERR_CUDA = 3,        /* a CUDA launch or runtime call failed */
    SQ_ERR_TIMEOUT = 4,     /* reserved: a bounded device wait gave up */
    SQ_ERR_NUMERIC = 5      /* a superquadric parameter outside its domain (device status only) */
} sq_status_t;

enum { SQ_INDEX_OBB = 0, SQ_INDEX_CUBE = 1, SQ_INDEX_OBB_OPACITY = 2 };
enum { SQ_OP_INDEX = 0, SQ_OP_FWD = 1, SQ_OP_BWD = 2, SQ_OP_QUERY = 3 };

/* Limits of this build. */
#define SQ_MAX_CLASSES 32 /* n_classes in [1, 32] */
#define SQ_MAX_SAMPLES 1024 /* L in [1, 1024] */

/* Axis-aligned voxel grid: cells [lo + i*vs, lo + (i+1)*vs), n* >= 1, vs > 0,
 * nx*ny*nz < 2^31.  The paper's grid is [-40,40]^2 x [-1,5.4] m at 0.4 m
 * (Sec. 4.1): 200 x 200 x 16. */
typedef struct {
    int nx, ny, nz;
    float lo[3];
    float vs[3];
} sq_grid_t;

/* Superquadric set S (Sec. 3.1).  Device FP32 arrays:
 *   means [n,3], quats [n,4] (any non-zero length), scales [n,3] (> 0),
 *   eps [n,2] = (eps1, eps2) in (0, 2] (the paper constrains [0.1, 2.0], Supp. A.9),
 *   opacity [n] (sigma), logits [n, n_classes] (c). */
typedef struct {
    const float* means;
    const float* quats;
    const float* scales;
    const float* eps;
    const float* opacity;
    const float* logits;
    int n;         /* >= 0 */
    int n_classes; /* 1 .. SQ_MAX_CLASSES */
    int sem_mode;  /* SQ_SEM_RAW: c_k as given (Eq. 4, the default); SQ_SEM_SOFTMAX:
                      c_k replaced by softmax(c_k) over the classes of each primitive
                      (g_logits are then w.r.t. the raw logits, through the softmax) */
} sq_prims_t;

enum { SQ_SEM_RAW = 0, SQ_SEM_SOFTMAX = 1 };

/* How a primitive's voxel neighbourhood is chosen (Sec. 3.3.1).
 *  SQ_INDEX_OBB:  the world AABB of the oriented box that holds the level set
 *                 p_o >= tau_cut (local half-extents s_i * ln(1/tau_cut)^(eps1/2)),
 *                 mapped to an inclusive voxel range.  tau_cut in (0, 1).
 *  SQ_INDEX_CUBE: the voxel holding the centre +- nv voxels per axis (the
 *                 paper's cubic neighbourhood N_v = 5, Sec. 4.2).  nv >= 0.
 *  SQ_INDEX_OBB_OPACITY: the opacity-aware refinement the paper names as future
 *                 work (Supp., limitations): as SQ_INDEX_OBB for the level set
 *                 sigma_i p_o >= tau_cut, local half-extents
 *                 s_i * (ln(sigma_i) - ln(tau_cut))^(eps1/2); a primitive with
 *                 sigma_i <= tau_cut is listed nowhere.  It drops only pair terms
 *                 whose sigma p_o is below tau_cut (their p_o c terms too). */
typedef struct {
    int mode;
    float tau_cut;
    int nv;
} sq_index_opts_t;

/* The voxel -> superquadric index (V_n, V_f, V_sq of Sec. 3.3.1), caller-owned
 * device buffers:
 *   v_n    [nvox] int32  number of primitives listed for each voxel
 *   v_f    [nvox] int32  offset of each voxel's list in v_sq (exclusive prefix sum of v_n)
 *   v_sq   [capacity] int32  primitive ids, each voxel's list ascending, no duplicates
 *   ranges [n,6] int32  per primitive (i0,i1,j0,j1,k0,k1) inclusive; empty = (0,-1,0,-1,0,-1)
 *   p_total  device int64 scalar: total entries P (written even on overflow)
 *   status   device int32 scalar after sq_build_index: SQ_OK; SQ_ERR_CAPACITY;
 *            or SQ_ERR_NUMERIC when a parameter of some primitive lies outside
 *            the domain sq_prims_t states (a NaN or infinity anywhere, a
 *            zero-length quaternion, a scale <= 0, eps outside (0, 2]), which
 *            takes precedence.  While it is non-zero v_sq is not written and the
 *            render and query kernels do no work (forward outputs stay as they
 *            were, gradients come out zero).
 * P must stay below 2^31. */
typedef struct {
    int* v_n;
    int* v_f;
    int* v_sq;
    int* ranges;
    long long capacity;
    long long* p_total;
    int* status;
    /* Optional (NULL = absent), no counterpart in the paper: [capacity] uint16,
     * for every entry of v_sq the position of its voxel v against the primitive's
     * voxel range (i0..i1, j0..j1, k0..k1) per axis a (bits 4a..4a+3):
     * lo_a == v_a, lo_a == v_a - 1, hi_a == v_a, hi_a == v_a + 1.  Written by
     * sq_build_index when non-NULL; sq_render_bwd uses it to find where a ray
     * enters a primitive's range without reading the range (faster backward). */
    unsigned short* v_flags;
} sq_index_t;

/* Rays and samples (Sec. 3.3.1): n_cam cameras of H x W pixels, L sample depths
 * t[L] (device FP32, the caller's spacing; the paper samples uniformly in
 * [t_near, t_far]), kappa = early-termination threshold on T (0 = none, the
 * paper's default, Sec. 4.2), alpha_max = upper bound of alpha (1 in the paper,
 * Sec. 3.3.2). */
typedef struct {
    int n_cam, H, W;
    const float* K;         /* [n_cam, 4] device */
    const float* cam2world; /* [n_cam, 3, 4] device */
    const float* t;         /* [L] device */
    int L;
    float kappa;
    float alpha_max;
} sq_rays_t;

/* Bytes of workspace an entry point needs (op = SQ_OP_*); rays may be NULL for
 * SQ_OP_INDEX, SQ_OP_FWD and SQ_OP_QUERY.  SQ_OP_QUERY needs the grid (the query
 * backward keeps the cotangent row of every voxel, padded to a multiple of 4
 * classes).  SQ_OP_BWD needs rays: besides the
 * per-primitive records it holds 8 bytes per sample of every ray (dL/dalpha_j
 * and w_j from the back-to-front sweep), 16 bytes per ray and per primitive and
 * camera, and up to 64 tile sums of 192 bytes and 64 queue entries per primitive
 * (the primitive-major order).  Returns 0 on invalid arguments. */
size_t sq_workspace_size(int op, const sq_prims_t* prims, const sq_grid_t* grid, const sq_rays_t* rays);

/* Sec. 3.3.1 "Preliminary Construction": per-primitive voxel ranges, V_n by a
 * count pass, V_f by an exclusive scan, V_sq sorted by id: written by voxel
 * tiles, each voxel appending in id order the primitives whose range holds it
 * (grids up to 65,535 voxels per axis), else by a scatter and a per-voxel sort.
 * Writes ranges, v_n, v_f, p_total, status and (when P <= capacity) v_sq.  On P > capacity, status = SQ_ERR_CAPACITY, v_sq is left partial and
 * p_total holds the needed capacity. */
sq_status_t sq_build_index(const sq_prims_t* prims, const sq_grid_t* grid, const sq_index_opts_t* opts,
                           sq_index_t* index, void* workspace, size_t workspace_bytes, void* stream);

/* The forward state that sq_render_fwd saves for sq_render_bwd.  Only the
 * samples a ray composites (up to its early stop) take memory: they are saved in
 * pages of SQ_SAVE_PAGE consecutive samples of one ray, handed out as the rays
 * advance, per sample (T_j, alpha_j) as FP32 (the transmittance before the
 * sample; alpha_j negated where the alpha_max clamp was active) and s_j as CP FP32
 * (Eq. 4; CP = n_classes rounded up to a multiple of 4, the padding zero).
 * Layout of the caller's buffer (each block 256-byte aligned): a 256-byte header
 * -- int64 at byte 0: the pages the last forward needed (written even when they
 * did not fit), int32 at byte 8: SQ_OK or SQ_ERR_CAPACITY --; the page of every
 * SQ_SAVE_PAGE samples of every ray [R, ceil(L / SQ_SAVE_PAGE)] int32; the
 * per-ray count of composited samples [R] int32; then as many pages as the
 * buffer holds.  When the pages run out the forward still writes its outputs,
 * sets SQ_ERR_CAPACITY and the header's page count, and a backward from that
 * state does no work (zero gradients): size the buffer again from the count
 * (sq_saved_size_pages) and rerun the forward.
 * sq_saved_size: the bytes for every sample of every ray (always enough).
 * sq_saved_size_pages: the bytes for a buffer of `pages` pages.
 * 0 on invalid rays, n_classes or pages. */
#define SQ_SAVE_PAGE 8
size_t sq_saved_size(const sq_rays_t* rays, int n_classes);
size_t sq_saved_size_pages(const sq_rays_t* rays, int n_classes, long long pages);

/* Sec. 3.3.2 forward pass (Eq. 2, 4-6).  Per ray r:
 *   depth[r]   = sum_j w_j t_j,                  w_j = T_j alpha_j, T_j = prod_{l<j} (1 - alpha_l)
 *   sem[r, :]  = sum_j w_j s_j,                  alpha_j = min(sum_k p_o sigma_k, alpha_max),
 *                                                 s_j = sum_k p_o c_k over k in Q(voxel of sample j)
 *   t_final[r] = transmittance after the last composited sample (nullable).
 * With kappa > 0 a ray stops after the first sample whose following T < kappa;
 * a ray also stops once T is exactly 0 (all later weights vanish).
 * t must be non-decreasing (the paper's uniform samples are): a ray that has
 * left the grid is not followed further.
 * Outputs: depth [R], sem [R, n_classes], t_final [R]; R = n_cam*H*W.
 * saved (nullable, caller-owned device memory of saved_bytes, at least
 * sq_saved_size_pages(rays, C, 1)) receives the state the backward pass needs
 * (see sq_saved_size); pass NULL for inference. */
sq_status_t sq_render_fwd(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                          const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* saved,
                          size_t saved_bytes, void* workspace, size_t workspace_bytes, void* stream);

/* No counterpart in the paper.  The forward render of sq_render_fwd for callers
 * that cannot allocate device memory when they render and have no workspace to
 * lend the library -- for instance a real-time loop that forbids allocation after
 * start-up (cudaMalloc can block and synchronise the device), or a plugin whose
 * host framework owns every device buffer.  Same arguments and outputs as
 * sq_render_fwd without saved state or workspace: the scratch comes from a
 * buffer built into the library (a static device array of about 7.4 MB, held on
 * every device that loads the library until exit).  Limits: prims->n at most
 * SQ_NOALLOC_MAX_PRIMS (otherwise SQ_ERR_INVALID_ARG, no work done).  The first
 * call on each device looks up the buffer's device address; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset on a device, do not call this entry point on
 * that device again.  All calls share the buffer, so calls that overlap on the
 * GPU race; order them (one stream, or events).  Allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library call -- unless kernel timing
 * is switched on (sq_profile_enable), which creates CUDA events as it records
 * launches; leave it off where nothing may be allocated. */
#define SQ_NOALLOC_MAX_PRIMS 16384
sq_status_t sq_render_fwd_noalloc(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                                  const sq_rays_t* rays, float* depth, float* sem, float* t_final, void* stream);

/* Sec. 3.3.3 backward pass: given dL/d depth [R] and dL/d sem [R, n_classes]
 * and the state a forward call with the same inputs saved, overwrites
 * g_means [n,3], g_quats [n,4] (w.r.t. the raw, unnormalised quaternion),
 * g_scales [n,3], g_eps [n,2], g_opacity [n], g_logits [n, C] with
 * dL/d(parameter).  Samples are swept back to front, so that
 * dL/dalpha_j = T_j (v_j - U_j) with v_j = gD t_j + <gS, s_j> and
 * U_j = alpha_{j+1} v_{j+1} + (1 - alpha_{j+1}) U_{j+1} needs no division by
 * (1 - alpha).  The index is treated as constant.  Where the alpha clamp is
 * active (sum > alpha_max) no gradient flows through that sample's alpha.
 * Accumulates in the default order (SQ_BWD_DEFAULT, below): primitive-major,
 * bitwise reproducible; sq_render_batched takes the order as a tuning field. */
sq_status_t sq_render_bwd(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                          const sq_rays_t* rays, const void* saved, size_t saved_bytes, const float* grad_depth,
                          const float* grad_sem, float* g_means, float* g_quats, float* g_scales, float* g_eps,
                          float* g_opacity, float* g_logits, void* workspace, size_t workspace_bytes, void* stream);

/* Batched rendering of many scenes (uneven primitive, camera, ray and sample
 * counts) in one persistent launch per pass: the rays of all scenes form one
 * range handed out by a global work counter, so a launch stays busy until the
 * last ray of the last scene.  The paper renders the 2T+1 frames of its temporal
 * horizon per training step (Sec. 3.2); here any set of scenes sharing
 * n_classes can be batched.  A scene carries what sq_render_fwd and
 * sq_render_bwd take: for SQ_OP_FWD depth/sem/t_final outputs and an optional
 * saved buffer; for SQ_OP_BWD the saved buffer written by the forward, the
 * cotangents and the six gradient outputs.  Only kernel launches and async
 * memsets are issued (the scene descriptors travel as kernel arguments), so a
 * call can be captured in a CUDA graph. */
#define SQ_MAX_BATCH 32
typedef struct {
    sq_prims_t prims;
    sq_index_t index;
    sq_grid_t grid;
    sq_rays_t rays;
    float* depth;        /* [R] forward outputs */
    float* sem;          /* [R, C] */
    float* t_final;      /* [R], nullable */
    void* saved;         /* sq_saved_size(&rays, n_classes) bytes; nullable for inference forwards */
    size_t saved_bytes;
    const float* grad_depth; /* [R] backward inputs */
    const float* grad_sem;   /* [R, C] */
    float* g_means;      /* backward outputs, as in sq_render_bwd */
    float* g_quats;
    float* g_scales;
    float* g_eps;
    float* g_opacity;
    float* g_logits;
    /* Optional diagnostic output (NULL = not wanted), no counterpart in the paper:
     * [prims.n] device int64.  An SQ_OP_BWD call in the primitive-major order
     * overwrites it with the number of (sample, primitive) pairs it evaluated for
     * each primitive: the samples j < (composited count of the ray) of every ray
     * whose voxel lies in the primitive's voxel range.  The ray-major order and
     * SQ_OP_FWD leave it untouched. */
    long long* pair_visits;
} sq_scene_t;

/* Order of the backward's gradient accumulation (Sec. 3.3.3).  Both first sweep
 * every ray back to front (Process 1: dL/dalpha_j and w_j per sample).
 *   SQ_BWD_RAY_MAJOR: a warp per pair of rays walks the rays' samples, one lane
 *     per (ray, primitive) run, and flushes each run's partial sums to the
 *     primitive with atomic adds (summation order varies between runs).
 *   SQ_BWD_PRIMITIVE_MAJOR: the paper's grouping (Processes 2-3): each
 *     primitive's interactions are generated from its voxel box (the pixels of
 *     its projected rectangle, the exact sample interval of each pixel's ray in
 *     the box), reduced per tile of candidate pixels by one CTA and summed over
 *     the tiles in a fixed order: no atomics, bitwise reproducible gradients.
 *   SQ_BWD_DEFAULT: the library's choice, primitive-major (the faster of the two
 *     on the six-camera frame; sq_autotune measures both on a given batch). */
enum { SQ_BWD_DEFAULT = 0, SQ_BWD_RAY_MAJOR = 1, SQ_BWD_PRIMITIVE_MAJOR = 2 };

/* Launch configuration: lanes (= samples marched together, the sample chunk)
 * per ray in the forward (4, 8 or 16), warps per CTA in the forward (1..8) and
 * in the ray-major backward (1..8, or 0: the count that keeps the most warps
 * resident for the batch's largest L, whose sample tables set the backward's
 * shared memory), the backward order (SQ_BWD_*), and the forward's ray tile: the
 * consecutive rays a lane group takes from the batch's work queue at a time
 * (1..64; 0 = 1).  The defaults are {4, 8, 0, SQ_BWD_DEFAULT, 1}. */
typedef struct {
    int fwd_lanes_per_ray;
    int fwd_warps_per_cta;
    int bwd_warps_per_cta;
    int bwd_order;
    int fwd_ray_tile;
} sq_tuning_t;

/* Workspace bytes for sq_render_batched / sq_autotune on these scenes; when
 * every scene has saved state it includes the backward's buffers (as for
 * SQ_OP_BWD in sq_workspace_size). */
size_t sq_batched_workspace_size(const sq_scene_t* scenes, int n_scenes);

/* op = SQ_OP_FWD or SQ_OP_BWD over n_scenes (1..SQ_MAX_BATCH) scenes; tuning
 * nullable (defaults).  Scenes must share n_classes. */
sq_status_t sq_render_batched(int op, const sq_scene_t* scenes, int n_scenes, const sq_tuning_t* tuning,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Autotuner: times every forward configuration (lanes per ray x warps per CTA x
 * ray tile) and, when every scene has saved state and cotangents, every backward
 * one on these scenes (reps timed launches each, CUDA events on the stream) and
 * writes the fastest to *best.  fwd_ms[8] / bwd_ms[4] (nullable) receive the
 * mean times of the candidates in the order {4,4,1},{4,8,1},{8,4,1},{8,8,1},
 * {4,4,16},{4,8,16},{8,4,16},{8,8,16} (lanes, warps, ray tile) and ray-major
 * with {0},{4},{8} warps per CTA (0 = automatic), then primitive-major.
 * Host-synchronous and overwrites the scenes' outputs; call it outside any
 * stream capture. */
sq_status_t sq_autotune(const sq_scene_t* scenes, int n_scenes, void* workspace, size_t workspace_bytes, void* stream,
                        int reps, sq_tuning_t* best, float* fwd_ms, float* bwd_ms);

/* Supp. A.4 voxelisation at every voxel centre p = lo + (i + 0.5) vs (FP32):
 *   density[v] = sum_{k in Q(v)} p_o(p, S_k) sigma_k, sem[v, :] = sum p_o c_k,
 *   label[v] = argmax_c sem[v, c] (lowest c on ties) if density >= tau, else
 *   n_classes ("free").  label is nullable (uint8, so n_classes <= 255).  Every
 *   voxel sums its list Q(v) in ascending id order; the sums are evaluated by
 *   voxel tiles (the primitives whose voxel range meets the tile, staged in
 *   shared memory) on grids up to 65,535 voxels per axis, else by lane groups
 *   merging neighbouring voxels' lists.  The index's ranges and lists are read. */
sq_status_t sq_query_grid(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid, float tau,
                          float* density, float* sem, unsigned char* label, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Backward of sq_query_grid (differentiable voxelisation, the next step the
 * paper's NYUv2 voxel losses ask for; Supp. A.4): given dL/d density [nvox] and
 * dL/d sem [nvox, n_classes] (device FP32, all voxels), overwrites g_means [n,3],
 * g_quats [n,4] (raw quaternion), g_scales [n,3], g_eps [n,2], g_opacity [n],
 * g_logits [n, n_classes] with dL/d(parameter), the index held fixed.  Per pair
 * (voxel v, k in Q(v)): dL/dp_o = gd[v] sigma_k + <gs[v], c_k>.  Labels are not
 * differentiable.  Workspace: sq_workspace_size(SQ_OP_QUERY, ...).  Runs no
 * work (zero gradients) while the index status is non-zero. */
sq_status_t sq_query_grid_bwd(const sq_prims_t* prims, const sq_index_t* index, const sq_grid_t* grid,
                              const float* grad_density, const float* grad_sem, float* g_means, float* g_quats,
                              float* g_scales, float* g_eps, float* g_opacity, float* g_logits, void* workspace,
                              size_t workspace_bytes, void* stream);

/* Training loss of Supp. A.5 (Eq. 8) and its gradient w.r.t. the rendered maps:
 *   L = lambda_s * mean_r CE(softmax(sem[r]), label[r]) + lambda_d * mean_r (depth[r] - target[r])^2.
 * Writes loss (device scalar, overwritten), grad_depth [R], grad_sem [R, C].
 * labels are int32 in [0, C); a label outside it makes the loss NaN (that ray's
 * gradient row then has no one-hot term).  n_classes in [1, SQ_MAX_CLASSES],
 * else SQ_ERR_INVALID_ARG. */
sq_status_t sq_loss_ce_mse(const float* depth, const float* sem, const float* target_depth, const int* target_label,
                           long long n_rays, int n_classes, float lambda_s, float lambda_d, float* loss,
                           float* grad_depth, float* grad_sem, void* stream);

/* Voxel losses of the grid query (Supp. A.4: cross-entropy on the semantic
 * voxels, binary cross-entropy on the density voxels).  Labels y[v], int32:
 * 0..C-1 an occupied voxel of that class, C a free voxel, -1 ignored.  With
 * occupancy probability p = 1 - exp(-d) of the density d >= 0 (the chance that
 * a ray through the voxel is absorbed, the compositing's alpha for density d):
 *   L = lambda_s * mean_{y in [0,C)} CE(softmax(sem[v]), y[v])
 *     + lambda_o * mean_{y in [0,C]} BCE(p[v], y[v] < C),
 * where BCE(p, 0) = d and BCE(p, 1) = -log(1 - exp(-max(d, 1e-6))) (no gradient
 * below the clamp).  Negative densities count as 0.  A mean over an empty set is
 * 0.  Writes loss[0..2] = (L, semantic term, occupancy term), counts[0..1] =
 * (occupied, labelled) voxels, grad_density [V], grad_sem [V, C] (all device,
 * overwritten; counts also serves the normalisation).  n_classes in
 * [1, SQ_MAX_CLASSES], else SQ_ERR_INVALID_ARG. */
sq_status_t sq_loss_voxel(const float* density, const float* sem, const int* label, long long n_voxels,
                          int n_classes, float lambda_s, float lambda_o, float* loss, int* counts,
                          float* grad_density, float* grad_sem, void* stream);

/* Work counter for throughput and roofline reports: out[0] = Q, the number of
 * (sample, primitive) pairs the forward pass evaluates (sum over in-grid
 * samples of V_n of the sample's voxel, all L samples, no early termination),
 * out[1] = number of in-grid samples.  out: device int64[2], overwritten. */
sq_status_t sq_count_pairs(const sq_index_t* index, const sq_grid_t* grid, const sq_rays_t* rays, long long* out,
                           void* stream);

const char* sq_status_string(sq_status_t status);

/* Human-readable text of the last SQ_ERR_* raised on the calling host thread. */
const char* sq_last_error(void);

/* Per-kernel timing, no counterpart in the paper.  While enabled, every kernel
 * the library launches is bracketed by two CUDA events recorded on its stream
 * (up to SQ_PROFILE_MAX_LAUNCHES launches; later ones are only counted as
 * dropped).  Enabling clears the records.  Meant for benchmarks on one device;
 * do not enable it while a stream is being captured into a graph. */
#define SQ_PROFILE_MAX_LAUNCHES 8192
sq_status_t sq_profile_enable(int on);

/* Host-synchronous: waits for the recorded events and returns the number of
 * recorded launches of kernel `name` (for example "k_backward"; NULL = every
 * kernel) and their summed duration in milliseconds; *dropped (nullable) gets
 * the number of launches that found the record pool full. */
sq_status_t sq_profile_query(const char* name, long long* launches, double* total_ms, long long* dropped);

/* Measured throughput of the special-function unit, no counterpart in the
 * paper: the renderer's pair kernels are bound by its exp2 / log2 / reciprocal
 * instructions (9 per pair in the forward, 13 in the backward), and a roofline
 * should divide by the rate this device reaches rather than a nominal count per
 * clock.  op: 0 = ex2.approx, 1 = lg2.approx, 2 = rcp.approx.  Runs a few
 * milliseconds of independent chains of that instruction on every SM (the
 * fastest of three timed launches, CUDA events on `stream`, host-synchronous)
 * and writes the instructions per second (all lanes) to *ops_per_s.  Creates
 * two CUDA events; allocates no device memory. */
sq_status_t sq_measure_sfu(int op, double* ops_per_s, void* stream);

/* Bounds checks of the debug build, no counterpart in the paper (the stand-in for a
 * memory checker).  The library built with -DSQR_CHECK (libsqr_check.so) checks the
 * indices its kernels take from caller-owned data before using them: a voxel list
 * (V_f, V_n) lying outside V_sq's capacity (site 1), a listed id that is not a
 * primitive (site 2), a saved-state page outside the saved buffer (site 3).  A failed
 * check skips the access and records its site in a device word; the kernel goes on
 * (no trap, no assert) and its outputs are then not meaningful.  Covered: the
 * forward render, the backward sweep, the ray-major backward's listed ids, and the
 * untiled grid query; the index build, the primitive-major backward and the tiled
 * query read only data the library derives itself.
 * sq_check_query writes 1 to *compiled when the loaded library has the checks (0
 * otherwise, and then *site = 0), and to *site the first failing site since the
 * last query (0: none), clearing it.  Host-synchronous (device-to-host copies). */
sq_status_t sq_check_query(int* compiled, int* site);

#ifdef __cplusplus
}
#endif

#endif /* SQR_H */
