// sqr_pair.cuh -- per-pair derivatives of the occupancy (Eq. 1-2) shared by the
// render backward and the grid-query backward.
#pragma once

#include "sqr_common.cuh"

namespace sqr {

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

// Adds one pair's weighted partials to running sums, with dL/dp_o = G sigma + w <gS, c>:
//   acc[0..10] += -p_o dL/dp_o r[i],  acc[11] += G p_o,  acc[12] += w p_o.
__device__ __forceinline__ void accumulate(float acc[13], float po, const float pr[11], float G, float w, float sigma,
                                           float cd) {
    const float gf = -po * fmaf(G, sigma, w * cd);
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = fmaf(gf, pr[i], acc[i]);
    acc[11] = fmaf(G, po, acc[11]);
    acc[12] = fmaf(w, po, acc[12]);
}

}  // namespace sqr
