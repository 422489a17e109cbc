// f32_device.cuh -- device helpers of the FP32-bulk PD substep shared by the
// sliced-ELL kernel and the lattice kernels: compensated pairs, the per-node
// time integration and the broken-bond counter.
#pragma once

#include "pd.h"

namespace pdmts {

// ------------------------------------------------------------- FP32 bulk --
// Compensated addition (hi, lo) += x: Knuth's two-sum followed by a
// renormalisation. Explicit round-to-nearest intrinsics keep the compiler
// from fusing the caller's product into the first sum, which would break the
// error term.
__device__ __forceinline__ void df_add(float &hi, float &lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    e = __fadd_rn(e, lo);
    const float h2 = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(h2, s));
    hi = h2;
}

template <int DIM>
__device__ __forceinline__ void load_pair(const float4 *p4, const float2 *p2, int64_t i, float (&h)[DIM],
                                          float (&l)[DIM])
{
    const float4 q = p4[i];
    if constexpr (DIM == 2) {
        h[0] = q.x; h[1] = q.y; l[0] = q.z; l[1] = q.w;
    } else {
        const float2 r = p2[i];
        h[0] = q.x; h[1] = q.y; h[2] = q.z; l[0] = q.w; l[1] = r.x; l[2] = r.y;
    }
}

template <int DIM>
__device__ __forceinline__ void store_pair(float4 *p4, float2 *p2, int64_t i, const float (&h)[DIM],
                                           const float (&l)[DIM])
{
    if constexpr (DIM == 2) {
        p4[i] = make_float4(h[0], h[1], l[0], l[1]);
    } else {
        p4[i] = make_float4(h[0], h[1], h[2], l[0]);
        p2[i] = make_float2(l[1], l[2]);
    }
}

// Per-node part of an FP32-bulk substep: a = (f + wb + theta g) / m,
// v += dt/2 (a_old + a), next prediction u + dt v + dt^2/2 a (lattice units).
template <int DIM>
__device__ __forceinline__ void finish_node_f32(const F32NodeArgs &N, const int64_t i, const float (&f)[DIM],
                                                float (&uh)[DIM], float (&ul)[DIM], const int init)
{
    const int64_t n = N.n;
    const float im = N.inv_m[i];
    float an[DIM], ao[DIM];
    if constexpr (DIM == 2) {
        const float2 q = reinterpret_cast<const float2 *>(N.a)[i];
        ao[0] = q.x; ao[1] = q.y;
    } else {
        const float4 q = reinterpret_cast<const float4 *>(N.a)[i];
        ao[0] = q.x; ao[1] = q.y; ao[2] = q.z;
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        float t = f[d];
        if (N.wb)
            t = __fadd_rn(t, N.wb[d * n + i]);
        if (N.g)
            t = __fmaf_rn(N.theta, N.g[d * n + i], t);
        an[d] = __fmul_rn(t, im);
    }
    float vh[DIM], vl[DIM];
    load_pair<DIM>(N.v4, N.v2, i, vh, vl);
    if (!init) {
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            df_add(vh[d], vl[d], __fmul_rn(N.hdt, __fadd_rn(ao[d], an[d])));
        store_pair<DIM>(N.v4, N.v2, i, vh, vl);
    }
    if constexpr (DIM == 2)
        reinterpret_cast<float2 *>(N.a)[i] = make_float2(an[0], an[1]);
    else
        reinterpret_cast<float4 *>(N.a)[i] = make_float4(an[0], an[1], an[2], 0.f);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
        df_add(uh[d], ul[d], __fmaf_rn(N.dt, vh[d], __fmaf_rn(N.dt, vl[d], __fmul_rn(N.hdt2, an[d]))));
    store_pair<DIM>(N.u4_out, N.u2_out, i, uh, ul);
}

// Packed FP32x2 forms: one instruction for both components, each rounded
// exactly like the scalar operation (a - b as fma(b, -1, a), rounded once).
__device__ __forceinline__ float2 fsub2(const float2 a, const float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 splat2(const float x) { return make_float2(x, x); }

// df_add on both components at once: the same operations as df_add.
__device__ __forceinline__ void df_add2(float2 &hi, float2 &lo, const float2 x)
{
    const float2 s = __fadd2_rn(hi, x);
    const float2 bp = fsub2(s, hi);
    float2 e = __fadd2_rn(fsub2(hi, fsub2(s, bp)), fsub2(x, bp));
    e = __fadd2_rn(e, lo);
    const float2 h2 = __fadd2_rn(s, e);
    lo = fsub2(e, fsub2(h2, s));
    hi = h2;
}

// finish_node_f32<2> with the node's inputs already at hand (staged in shared
// memory), both components in packed FP32x2: the same operations in the same
// order per component, so the same bits.
__device__ __forceinline__ void finish_node_2d_vals(const F32NodeArgs &N, const int64_t i, const float (&f)[2],
                                                    float (&uh)[2], float (&ul)[2], const float2 ao,
                                                    const float4 vv, const float im, const float2 wb,
                                                    const float2 g, const int init)
{
    float2 t = make_float2(f[0], f[1]);
    if (N.wb)
        t = __fadd2_rn(t, wb);
    if (N.g)
        t = __ffma2_rn(splat2(N.theta), g, t);
    const float2 an = __fmul2_rn(t, splat2(im));
    float2 vh = make_float2(vv.x, vv.y), vl = make_float2(vv.z, vv.w);
    if (!init) {
        df_add2(vh, vl, __fmul2_rn(splat2(N.hdt), __fadd2_rn(ao, an)));
        N.v4[i] = make_float4(vh.x, vh.y, vl.x, vl.y);
    }
    reinterpret_cast<float2 *>(N.a)[i] = an;
    float2 h = make_float2(uh[0], uh[1]), l = make_float2(ul[0], ul[1]);
    df_add2(h, l, __ffma2_rn(splat2(N.dt), vh, __ffma2_rn(splat2(N.dt), vl, __fmul2_rn(splat2(N.hdt2), an))));
    N.u4_out[i] = make_float4(h.x, h.y, l.x, l.y);
    uh[0] = h.x;
    uh[1] = h.y;
    ul[0] = l.x;
    ul[1] = l.y;
}

__device__ __forceinline__ void count_broken(unsigned long long *counter, unsigned nbroken)
{
    if (counter) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, nbroken);
        if ((threadIdx.x & 31) == 0 && tot)
            atomicAdd(counter, (unsigned long long)tot);
    }
}

// Weight of bond (i, j) in the Arlequin overlap: 1 - (alpha_i + alpha_j) / 2.
__device__ __forceinline__ float bond_weight(const float ai, const float aj)
{
    return __fmaf_rn(-0.5f, __fadd_rn(ai, aj), 1.f);
}

}  // namespace pdmts
