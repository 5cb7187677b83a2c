// sqr_render.cuh -- internal interface between the render translation units:
// per-scene descriptors (one or many scenes per launch), the packed-record
// layout, and the kernel launchers implemented in sqr_fwd.cu, sqr_bwd.cu and
// sqr_bwd_pm.cu.
#pragma once

#include "sqr_common.cuh"

namespace sqr {

constexpr int MAX_BATCH = 32;  // scenes per launch (= SQ_MAX_BATCH)
constexpr int SAVE_PS = SQ_SAVE_PAGE;  // samples per page of the saved forward state
constexpr int GF = 48;         // floats per primitive in the gradient accumulator (12 partials + up to 32 classes)
constexpr int NRAW = 12;       // summed partials: gx 3, tau 3, u df/du 3, eps 2, sigma 1
constexpr int MAX_WARPS = 8;   // warps per CTA accepted by the render kernels

// Everything a render kernel needs about one scene.  Built on the host, written
// to device memory by k_write_desc (a by-value kernel argument, so batched
// launches stay capturable in a CUDA graph without host copies).
struct SceneDesc {
    const float4* rec;   // [N, REC4] packed forward records
    const float4* aux;   // [N, AUX4] backward extras
    const float* lpad;   // [N, CP] logits padded to CP
    const int4* boxes;   // [N] packed voxel boxes (backward)
    const int* v_n;
    const int* v_f;
    const int* v_sq;
    long long v_cap;     // entries V_sq holds (the bounds checks of the debug build)
    const unsigned short* v_flags;  // nullable: per-entry range-boundary flags
    const int* status;
    GridC g;
    const float* K;
    const float* c2w;
    const float* t;
    int n_cam, H, W, L, C, n;
    int sem_mode;        // SQ_SEM_*: the logit gradient goes through the softmax
    int cp;              // C padded to a multiple of 4 (lpad row length)
    long long R;
    float kappa, alpha_max;
    float* depth;        // forward outputs
    float* sem;
    float* t_final;
    // Saved forward state, in pages of SAVE_PS consecutive samples of one ray handed
    // out on demand, so that only the composited samples take memory:
    float2* save_TA;     // [cap * SAVE_PS] (T_j before the sample, alpha_j negated where clamped); nullable
    float4* save_S;      // [cap * SAVE_PS, CP/4] semantic vector s_j of each sample, zero-padded to CP
    int* save_n;         // [R] samples composited
    int* save_page;      // [R, save_np] page of samples SAVE_PS*i .. SAVE_PS*i+SAVE_PS-1 of each ray
    unsigned long long* save_ctr;  // pages handed out (the pages the forward needed, even past cap)
    int* save_status;    // SQ_OK, or SQ_ERR_CAPACITY once a page request found no room
    long long save_cap;  // pages the buffer holds
    int save_np;         // pages per ray, ceil(L / SAVE_PS)
    float2* gw;          // [R, L] backward: (dL/dalpha_j, w_j) from the sweep
    const float* grad_depth;  // backward inputs
    const float* grad_sem;
    float* gacc;         // [N, GF] gradient accumulator (zeroed per backward)
    int4* pm_rect;       // [N, n_cam] primitive-major backward: pixel rectangle (u0, v0, u1, v1) of each box
    float4* pm_dir;      // [R] primitive-major backward: ray direction of each pixel, composited samples in .w
    long long* pair_visits;  // [N] nullable: (sample, primitive) pairs the primitive-major backward evaluated
    float4* pm_gs;       // [R, CP/4] primitive-major backward: grad_sem rows zero-padded to CP classes
};

struct BatchParams {
    int n;
    long long off[MAX_BATCH + 1];   // ray offsets of the scenes in the concatenated ray range
    long long boff[MAX_BATCH + 1];  // offsets of the scenes' ray bundles (backward)
    long long gboff[2 * MAX_BATCH];  // the same per launch group of the backward, from the group's first scene
    SceneDesc s[MAX_BATCH];
};

// What the render kernels receive: descriptors and offsets in device memory and
// a zeroed work counter over the concatenated rays (or ray bundles).  A backward
// launch may cover a slice of the scenes: d then points at its first scene and
// boff at bundle offsets counted from that scene.
struct Batch {
    const SceneDesc* d;
    const long long* off;
    const long long* boff;
    int n;
    long long total;
    int* ctr;
    int lmax;  // largest L of the batch
    int ray_tile = 1;  // forward: consecutive rays a lane group takes from the work counter at a time
};

__device__ __forceinline__ int scene_of(const Batch& B, long long g) {
    int lo = 0, hi = B.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(B.off + mid) <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void scene_ray(const SceneDesc& S, long long r, float o[3], float d[3]) {
    const long long hw = (long long)S.H * S.W;
    const int cam = (int)(r / hw);
    const long long pix = r - (long long)cam * hw;
    const int v = (int)(pix / S.W), u = (int)(pix - (long long)v * S.W);
    pixel_ray(S.K + 4 * cam, S.c2w + 12 * cam, u, v, o, d);
}

// Launch configuration picked by the autotuner (or the defaults).
struct Tuning {
    int fwd_lanes;  // lanes (samples) per ray in the forward: 4, 8 or 16
    int fwd_warps;  // warps per CTA, forward: 4 or 8
    int bwd_warps;  // warps per CTA, ray-major backward: 1..8, or 0 for the count that keeps the most warps resident
    int bwd_order;  // SQ_BWD_RAY_MAJOR or SQ_BWD_PRIMITIVE_MAJOR
    int fwd_tile;   // consecutive rays a forward lane group takes from the work queue at a time
};

// Primitive-major backward (Sec. 3.3.3, Processes 2-3): the primitives of all
// scenes of a batch are numbered g = poff[scene] + k; each has cnt[g] candidate
// pixels (its box's rectangles), cut into at most PM_MAXT tiles whose partial
// sums land in part[tile, GF] and are reduced per primitive in tile order.
constexpr int PM_MAXT = 64;         // tiles per primitive at most
constexpr int PM_CHUNK = 512;       // candidate pixels a tile block takes per pass
constexpr int PM_TILE_CHUNKS = 8;   // passes per tile, unless the primitive would need more than PM_MAXT tiles

// The tiles are taken in a spatial order (queue position -> tile in qtile): the
// primitives' box centres sorted into PM_CELLS Morton cells per scene, so that the
// blocks resident at one time work on neighbouring primitives, whose runs lie on
// the same rays and samples and share their (dL/dalpha_j, w_j) lines in L2.  The
// order decides only which block sums a tile when; every tile's sum, and the
// tile-ordered sum per primitive, is the same whatever the order.
__host__ __device__ constexpr int pm_cell_bits(int a) { return a == 2 ? 2 : 5; }  // Morton cells per axis: 32 x 32 x 4
constexpr int PM_CELLS = 1 << 12;
constexpr int PM_VISIT_SLOT = GF - 1;  // tile row slot holding the tile's pair count (int bits); unused by sums

struct PmArgs {
    const long long* poff;  // [n_scenes + 1] primitive offsets of the scenes
    int nscene;             // scenes of the batch
    int ntot;               // primitives of all scenes
    int* cnt;               // [ntot] candidate pixels
    int* toff;              // [ntot + 1] tile offsets (exclusive scan of the tile counts)
    float* part;            // [ntot * PM_MAXT, GF] tile partial sums
    int* tprim;             // [ntot * PM_MAXT] primitive of each tile
    int* ctr;               // zeroed tile counter
    int* key;               // [ntot] Morton cell of each primitive's box centre
    int* qtile;             // [ntot * PM_MAXT] tile at each queue position
};

int device_sm_count();
int bwd_rays_per_bundle();
sq_status_t launch_forward(const Batch& B, int cp, const Tuning& tn, cudaStream_t st);
sq_status_t launch_sweep(const Batch& B, int cp, cudaStream_t st);
sq_status_t launch_backward(const Batch& B, int cp, const Tuning& tn, cudaStream_t st);
sq_status_t launch_backward_pm(const Batch& B, const PmArgs& A, int cp, cudaStream_t st);
sq_status_t launch_grad_out(const SceneDesc& S, float* gm, float* gq, float* gs, float* ge, float* go, float* gl,
                            cudaStream_t st);
sq_status_t launch_pack_boxes(const int* ranges, int n, int4* boxes, cudaStream_t st);

}  // namespace sqr
