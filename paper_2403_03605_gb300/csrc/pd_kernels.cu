// pd_kernels.cu -- the PD substep (hot path) for sm_103a.
//
// One thread per PD node, one warp per tile of 32 consecutive nodes. The
// family is a sliced-ELL layout with slice height 32: slot k of the 32 nodes
// of a tile is one coalesced 128-byte row, and on a lattice the 32 neighbours
// read in one slot are 32 consecutive nodes, so the neighbour gather is
// coalesced as well. Each node accumulates its own force in registers in
// ascending neighbour order: no atomics, no reductions, a fixed summation
// order. The broken-bond state is one bit per slot (uint32 words, 32 slots per
// word per node), cleared irreversibly and written back only when it changes.
//
// Per substep (arXiv 2403.03605, Eq. 1-4, Eq. 33-34, Eq. 38 with gamma = 1/2,
// beta = 0, and the free-problem interface term of Eq. 48a):
//   for each intact bond: xi, eta, breaking test s >= s0, force sum
//   a = (f + (1 - alpha) b + theta g) / ((1 - alpha) rho)
//   v += dt/2 (a_old + a);   u_next = u + dt v + dt^2/2 a   (next substep's u)
//
// Two precisions:
//  * FP64: the parity build. Every operation is IEEE FP64 with explicit
//    round-to-nearest intrinsics (no FMA contraction) in exactly the order of
//    the CPU oracle, so results and broken-bond sets are bit-identical.
//  * FP32 bulk: bond kinematics and forces in FP32 from displacement
//    differences in lattice units; u and v are compensated (hi + lo) FP32
//    pairs so differences keep ~48 bits; the per-bond family word packs the
//    neighbour index and a stencil id whose offset, micromodulus and
//    threshold sit in shared memory. No FP64 instruction in the bond loop.
#include <algorithm>
#include "f32_device.cuh"

namespace pdmts {

// ------------------------------------------------------------------ FP64 --
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

template <int DIM>
__global__ void __launch_bounds__(256) k_pd_step_f64(const F64StepArgs A, const int init)
{
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= A.fam.ntiles)
        return;
    const int64_t n = A.fam.n;
    const int64_t i = tile * 32 + lane;
    const bool valid = i < n;
    const int64_t ii = valid ? i : n - 1;
    const int K = A.fam.tile_k[tile];
    const int64_t base = A.fam.tile_ptr[tile];
    const int64_t mbase = A.fam.mask_ptr[tile];

    double xi_i[DIM], ui[DIM], f[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        xi_i[d] = A.X[d * n + ii];
        ui[d] = A.u_in[d * n + ii];
        f[d] = 0.0;
    }
    const double ai = A.alpha ? A.alpha[ii] : 0.0;
    unsigned nbroken = 0;

    for (int w = 0; 32 * w < K; ++w) {
        const uint32_t m0 = valid ? A.fam.mask[mbase + 32 * w + lane] : 0u;
        uint32_t m = m0;
        const int kend = min(32, K - 32 * w);
        for (int kk = 0; kk < kend; ++kk) {
            if (!((m0 >> kk) & 1u))
                continue;
            const int64_t slot = base + (int64_t)(32 * w + kk) * 32 + lane;
            const int64_t j = A.fam.col[slot];
            double xi[DIM], eta[DIM];
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                xi[d] = dsub(A.X[d * n + j], xi_i[d]);
                eta[d] = dsub(A.u_in[d * n + j], ui[d]);
            }
            double xi2 = 0.0, y2 = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d)
                xi2 = dadd(xi2, dmul(xi[d], xi[d]));
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const double y = dadd(xi[d], eta[d]);
                y2 = dadd(y2, dmul(y, y));
            }
            if (A.breaking && y2 >= dmul(A.s0p2, xi2)) {  // s >= s0 (Eq. 3-4)
                m &= ~(1u << kk);
                continue;
            }
            double wc = A.cb[slot];
            if (A.alpha) {
                const double w_ij = dsub(1.0, dmul(0.5, dadd(ai, A.alpha[j])));
                wc = dmul(w_ij, wc);
            }
            if (A.pmb) {
                const double r = __dsqrt_rn(xi2), ry = __dsqrt_rn(y2);
                const double s = ddiv(dsub(ry, r), r);
                const double cp = dmul(dmul(A.cb[slot], xi2), r);
                double wcp = cp;
                if (A.alpha)
                    wcp = dmul(dsub(1.0, dmul(0.5, dadd(ai, A.alpha[j]))), cp);
                const double sc = dmul(ddiv(dmul(wcp, s), ry), A.V[j]);
#pragma unroll
                for (int d = 0; d < DIM; ++d)
                    f[d] = dadd(f[d], dmul(sc, dadd(xi[d], eta[d])));
            } else {
                double dot = 0.0;
#pragma unroll
                for (int d = 0; d < DIM; ++d)
                    dot = dadd(dot, dmul(xi[d], eta[d]));
                const double sc = dmul(dmul(wc, dot), A.V[j]);
#pragma unroll
                for (int d = 0; d < DIM; ++d)
                    f[d] = dadd(f[d], dmul(sc, xi[d]));
            }
        }
        if (m != m0) {
            A.fam.mask[mbase + 32 * w + lane] = m;
            nbroken += __popc(m0 ^ m);
        }
    }
    if (A.broken) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, nbroken);
        if (lane == 0 && tot)
            atomicAdd(A.broken, (unsigned long long)tot);
    }
    if (!valid)
        return;
    const double mi = A.mass[i];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        double t = f[d];
        if (A.wb)
            t = dadd(t, A.wb[d * n + i]);
        if (A.g)
            t = dadd(t, dmul(A.theta, A.g[d * n + i]));
        const double an = ddiv(t, mi);
        double v = A.v[d * n + i];
        if (!init) {
            v = dadd(v, dmul(A.hdt, dadd(A.a[d * n + i], an)));
            A.v[d * n + i] = v;
        }
        A.a[d * n + i] = an;
        A.u_out[d * n + i] = dadd(dadd(ui[d], dmul(A.dt, v)), dmul(A.hdt2, an));
    }
}

// One bond of the FP32 path, in lattice units (offset d, relative
// displacement eta = u_j - u_i). Written once for both FP32 kernels with
// explicit round-to-nearest intrinsics, so the two produce identical bits:
//   lhs = 2 d.eta + |eta|^2  (= (|xi + eta|^2 - |xi|^2) / h^2, no cancellation)
//   breaks when lhs >= thr = s0 (2 + s0) |d|^2        (s >= s0, Eq. 3-4)
//   linear force  coef (d.eta) d ; PMB  coef |d|^2 lhs / ((|d+eta| + |d|)|d+eta|) (d + eta)
// Every expression is invariant under (d, eta) -> (-d, -eta), so bond (i, j)
// and (j, i) reach the same decision. `on` is the bond's intact bit; the
// evaluation is branch-free (a broken or absent bond contributes 0).
struct Bond2 {
    float2 nuh, nul;  // -u_i (hi, lo)
};

__device__ __forceinline__ void bond_2d(const float4 uj, const Bond2 &B, const float d0, const float d1,
                                        const float coef, const float thr, const float r2, const float rd,
                                        const bool on, const int breaking, const int pmb, const uint32_t bit,
                                        uint32_t &m, float2 &f)
{
    const float2 eh = __fadd2_rn(make_float2(uj.x, uj.y), B.nuh);
    const float2 el = __fadd2_rn(make_float2(uj.z, uj.w), B.nul);
    const float2 eta = __fadd2_rn(eh, el);
    const float dot = __fmaf_rn(d1, eta.y, __fmul_rn(d0, eta.x));
    const float e2 = __fmaf_rn(eta.y, eta.y, __fmul_rn(eta.x, eta.x));
    const float lhs = __fmaf_rn(2.f, dot, e2);
    const bool brk = on && breaking && lhs >= thr;
    m = brk ? (m & ~bit) : m;
    const float w = (on && !brk) ? coef : 0.f;
    if (!pmb) {
        const float sc = __fmul_rn(w, dot);
        f = __ffma2_rn(make_float2(sc, sc), make_float2(d0, d1), f);
    } else {
        const float ry = __fsqrt_rn(__fadd_rn(r2, fmaxf(lhs, -r2)));
        const float den = __fmul_rn(__fadd_rn(ry, rd), ry);
        const float sc = w != 0.f ? __fdiv_rn(__fmul_rn(__fmul_rn(w, r2), lhs), den) : 0.f;
        f = __ffma2_rn(make_float2(sc, sc), __fadd2_rn(make_float2(d0, d1), eta), f);
    }
}

template <int DIM>
__device__ __forceinline__ float bond_dot(const float (&d)[3], const float (&eta)[DIM])
{
    float dot = __fmul_rn(d[0], eta[0]);
#pragma unroll
    for (int k = 1; k < DIM; ++k)
        dot = __fmaf_rn(d[k], eta[k], dot);
    return dot;
}

template <int DIM>
__device__ __forceinline__ float eta_sq(const float (&eta)[DIM])
{
    float e2 = __fmul_rn(eta[0], eta[0]);
#pragma unroll
    for (int k = 1; k < DIM; ++k)
        e2 = __fmaf_rn(eta[k], eta[k], e2);
    return e2;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_pd_step_f32(const F32StepArgs A, const int init)
{
    __shared__ float4 s_d[kMaxStencil];  // {d0, d1, d2, coef}
    __shared__ float4 s_t[kMaxStencil];  // {thr, rd, r2, 0}
    for (int q = threadIdx.x; q < A.n_stencil; q += blockDim.x) {
        const StencilEntry e = A.stencil[q];
        s_d[q] = make_float4(e.d[0], e.d[1], e.d[2], e.coef);
        s_t[q] = make_float4(e.thr, e.rd, e.r2, 0.f);
    }
    __syncthreads();

    const F32NodeArgs &N = A.nd;
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= A.fam.ntiles)
        return;
    const int64_t n = A.fam.n;
    const int64_t i = tile * 32 + lane;
    const bool valid = i < n;
    const int64_t ii = valid ? i : n - 1;
    const int K = A.fam.tile_k[tile];
    const int64_t base = A.fam.tile_ptr[tile];
    const int64_t mbase = A.fam.mask_ptr[tile];
    const uint32_t *col = reinterpret_cast<const uint32_t *>(A.fam.col);

    float uh[DIM], ul[DIM], f[DIM];
    load_pair<DIM>(N.u4_in, N.u2_in, ii, uh, ul);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
        f[d] = 0.f;
    const float ai = A.alpha ? A.alpha[ii] : 0.f;
    Bond2 B;
    if constexpr (DIM == 2) {
        B.nuh = make_float2(-uh[0], -uh[1]);
        B.nul = make_float2(-ul[0], -ul[1]);
    }
    float2 f2 = make_float2(0.f, 0.f);
    unsigned nbroken = 0;

    for (int w = 0; 32 * w < K; ++w) {
        const uint32_t m0 = valid ? A.fam.mask[mbase + 32 * w + lane] : 0u;
        uint32_t m = m0;
        const int kend = min(32, K - 32 * w);
        const uint32_t *cp = col + base + (int64_t)(32 * w) * 32 + lane;
#pragma unroll 4
        for (int kk = 0; kk < kend; ++kk) {
            const uint32_t cw = __ldg(cp + 32 * kk);
            const uint32_t bit = 1u << kk;
            if (!(m0 & bit))
                continue;
            const uint32_t j = cw >> 8;
            const uint32_t sid = cw & 255u;
            const float4 sd = s_d[sid];
            const float4 st = s_t[sid];
            float coef = sd.w;
            if (A.alpha)
                coef = __fmul_rn(coef, bond_weight(ai, A.alpha[j]));
            if constexpr (DIM == 2) {
                bond_2d(N.u4_in[j], B, sd.x, sd.y, coef, st.x, st.z, st.y, true, N.breaking, N.pmb, bit, m, f2);
            } else {
                float jh[DIM], jl[DIM], eta[DIM];
                load_pair<DIM>(N.u4_in, N.u2_in, j, jh, jl);
#pragma unroll
                for (int d = 0; d < DIM; ++d)
                    eta[d] = __fadd_rn(__fsub_rn(jh[d], uh[d]), __fsub_rn(jl[d], ul[d]));
                const float dd[3] = {sd.x, sd.y, sd.z};
                const float dot = bond_dot<DIM>(dd, eta);
                const float lhs = __fmaf_rn(2.f, dot, eta_sq<DIM>(eta));
                if (N.breaking && lhs >= st.x) {
                    m &= ~bit;
                    continue;
                }
                if (N.pmb) {
                    const float ry = __fsqrt_rn(__fadd_rn(st.z, fmaxf(lhs, -st.z)));
                    const float sc = __fdiv_rn(__fmul_rn(__fmul_rn(coef, st.z), lhs),
                                               __fmul_rn(__fadd_rn(ry, st.y), ry));
#pragma unroll
                    for (int d = 0; d < DIM; ++d)
                        f[d] = __fmaf_rn(sc, __fadd_rn(dd[d], eta[d]), f[d]);
                } else {
                    const float sc = __fmul_rn(coef, dot);
#pragma unroll
                    for (int d = 0; d < DIM; ++d)
                        f[d] = __fmaf_rn(sc, dd[d], f[d]);
                }
            }
        }
        if (m != m0) {
            A.fam.mask[mbase + 32 * w + lane] = m;
            nbroken += __popc(m0 ^ m);
        }
    }
    if constexpr (DIM == 2) {
        f[0] = f2.x;
        f[1] = f2.y;
    }
    count_broken(N.broken, nbroken);
    if (!valid)
        return;
    finish_node_f32<DIM>(N, i, f, uh, ul, init);
}

// ----------------------------------------------------------- damage (Eq. 5)
__global__ void k_damage(const SellView fam, const int packed, const double *__restrict__ V,
                         double *__restrict__ phi)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= fam.n)
        return;
    const int64_t t = i >> 5, lane = i & 31;
    const int dg = fam.deg[i];
    const int64_t base = fam.tile_ptr[t], mbase = fam.mask_ptr[t];
    double num = 0.0, den = 0.0;
    for (int k = 0; k < dg; ++k) {
        uint32_t cw = (uint32_t)fam.col[base + (int64_t)k * 32 + lane];
        int64_t j = packed ? (int64_t)(cw >> 8) : (int64_t)cw;
        const uint32_t w = fam.mask[mbase + 32 * (k >> 5) + lane];
        den = __dadd_rn(den, V[j]);
        if ((w >> (k & 31)) & 1u)
            num = __dadd_rn(num, V[j]);
    }
    phi[i] = den > 0.0 ? __dsub_rn(1.0, __ddiv_rn(num, den)) : 0.0;
}

__global__ void k_damage_lattice(const int64_t n, const uint32_t *__restrict__ mask,
                                 const uint32_t *__restrict__ exists, const int words, double *__restrict__ phi)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int intact = 0, total = 0;
    for (int w = 0; w < words; ++w) {
        intact += __popc(mask[(int64_t)w * n + i]);
        total += __popc(exists[(int64_t)w * n + i]);
    }
    phi[i] = total > 0 ? 1.0 - (double)intact / (double)total : 0.0;
}

__global__ void k_unpack(const int dim, const int64_t n, const float4 *__restrict__ p4,
                         const float2 *__restrict__ p2, const int accel, const double h,
                         double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    if (accel) {
        if (dim == 2) {
            const float2 q = reinterpret_cast<const float2 *>(p4)[i];
            out[i] = (double)q.x * h;
            out[n + i] = (double)q.y * h;
        } else {
            const float4 q = p4[i];
            out[i] = (double)q.x * h;
            out[n + i] = (double)q.y * h;
            out[2 * n + i] = (double)q.z * h;
        }
        return;
    }
    const float4 q = p4[i];
    if (dim == 2) {
        out[i] = ((double)q.x + (double)q.z) * h;
        out[n + i] = ((double)q.y + (double)q.w) * h;
    } else {
        const float2 r = p2[i];
        out[i] = ((double)q.x + (double)q.w) * h;
        out[n + i] = ((double)q.y + (double)r.x) * h;
        out[2 * n + i] = ((double)q.z + (double)r.y) * h;
    }
}

// (1 - alpha) b for the FP64 path, (1 - alpha) b / h for the FP32 path, or
// only a finiteness check of b (flag set to 1 on NaN/Inf).
__global__ void k_weighted_load(const int dim, const int64_t n, const double *__restrict__ b,
                                const double *__restrict__ alpha64, const float *__restrict__ alpha32,
                                const double inv_h, double *__restrict__ wb64, float *__restrict__ wb32,
                                unsigned long long *flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    for (int d = 0; d < dim; ++d) {
        const double x = b[d * n + i];
        if (flag) {
            if (!isfinite(x))
                atomicExch(flag, 1ull);
            continue;
        }
        if (wb64)
            wb64[d * n + i] = alpha64 ? __dmul_rn(__dsub_rn(1.0, alpha64[i]), x) : x;
        if (wb32) {
            const double w = alpha32 ? 1.0 - (double)alpha32[i] : 1.0;
            wb32[d * n + i] = (float)(w * x * inv_h);
        }
    }
}

// ------------------------------------------------------- MTS helpers ------
__global__ void k_interface_force(const int dim, const int64_t n, const int64_t n_ov, const int32_t *__restrict__ ov_node,
                                  const int32_t *__restrict__ ov_k, const double *__restrict__ ov_N, const int corners,
                                  const double *__restrict__ lam, const int64_t nl, const double inv_h,
                                  double *__restrict__ g64, float *__restrict__ g32, double *__restrict__ g64b,
                                  float *__restrict__ g32b)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_ov)
        return;
    const int64_t p = ov_node[q];
    for (int d = 0; d < dim; ++d) {
        double g = 0.0;
        for (int a = 0; a < corners; ++a)
            g += ov_N[q * corners + a] * lam[d * nl + ov_k[q * corners + a]];
        if (g64)
            g64[d * n + p] = g;
        if (g32)
            g32[d * n + p] = (float)(g * inv_h);
        if (g64b)
            g64b[d * n + p] = g;
        if (g32b)
            g32b[d * n + p] = (float)(g * inv_h);
    }
}

__global__ void k_constraint(const int dim, const int64_t nl, const int64_t *__restrict__ gpd_ptr,
                             const int32_t *__restrict__ gpd_col, const double *__restrict__ gpd_val, const int64_t npd,
                             const double *__restrict__ v64, const float4 *__restrict__ v4,
                             const float2 *__restrict__ v2, const double h, const int32_t *__restrict__ gfe_col,
                             const double *__restrict__ gfe_val, const int gfe_w, const int64_t nfe,
                             const double *__restrict__ vfe, const double sign_pd, const double sign_fe,
                             double *__restrict__ y, const int64_t v4_stride, const int64_t y_stride,
                             float2 *__restrict__ yf)
{
    // one warp per multiplier node k, all components (rows c nl + k): the PD
    // velocities of the node's support are gathered once for every component;
    // blockIdx.y picks one of several FP32 velocity fields (v4 + y v4_stride)
    // and its output rows (y + y y_stride)
    v4 += (int64_t)blockIdx.y * v4_stride;
    y += (int64_t)blockIdx.y * y_stride;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nl)
        return;
    double sp[3] = {0.0, 0.0, 0.0};
    const int64_t e1 = gpd_ptr[k + 1];
#pragma unroll 4
    for (int64_t e = gpd_ptr[k] + lane; e < e1; e += 32) {
        const int64_t p = gpd_col[e];
        const double g = gpd_val[e];
        double vp[3];
        if (v64) {
            for (int c = 0; c < dim; ++c)
                vp[c] = v64[(int64_t)c * npd + p];
        } else {
            const float4 q = v4[p];
            if (dim == 2) {
                vp[0] = ((double)q.x + (double)q.z) * h;
                vp[1] = ((double)q.y + (double)q.w) * h;
            } else {
                const float2 q2 = v2[p];
                vp[0] = ((double)q.x + (double)q.w) * h;
                vp[1] = ((double)q.y + (double)q2.x) * h;
                vp[2] = ((double)q.z + (double)q2.y) * h;
            }
        }
        for (int c = 0; c < dim; ++c)
            sp[c] += g * vp[c];
    }
    for (int c = 0; c < dim; ++c) {
        double sf = 0.0;
        if (gfe_col && lane < gfe_w)
            sf = gfe_val[k * gfe_w + lane] * vfe[(int64_t)c * nfe + gfe_col[k * gfe_w + lane]];
        double t = sign_pd * sp[c] + sign_fe * sf;
        for (int o = 16; o > 0; o >>= 1)
            t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) {
            y[(int64_t)c * nl + k] = t;
            if (yf) {
                const float hi = __double2float_rn(t);
                yf[(int64_t)c * nl + k] = make_float2(hi, __double2float_rn(t - (double)hi));
            }
        }
    }
}

// U_PD += W and the next prediction for link-segment entry t (< seg_n[0] + seg_n[1]).
__device__ __forceinline__ void pd_add_link_node(const PDAddLink &A, const int64_t t)
{
    const int64_t i = t < A.seg_n[0] ? A.seg_lo[0] + t : A.seg_lo[1] + (t - A.seg_n[0]);
    const int64_t n = A.n;
    if (A.u) {
        for (int d = 0; d < A.dim; ++d) {
            const int64_t q = d * n + i;
            const double u = A.u[q] + A.wu[q], v = A.v[q] + A.wv[q], a = A.a[q] + A.wa[q];
            A.u[q] = u;
            A.v[q] = v;
            A.a[q] = a;
            A.u_pred[q] = u + A.dt * v + A.hdt2 * a;
        }
        return;
    }
    float uh[3], ul[3], vh[3], vl[3], wuh[3], wul[3], wvh[3], wvl[3], a[3];
    if (A.dim == 2) {
        load_pair<2>(A.u4, A.u2, i, reinterpret_cast<float(&)[2]>(uh), reinterpret_cast<float(&)[2]>(ul));
        load_pair<2>(A.v4, A.v2, i, reinterpret_cast<float(&)[2]>(vh), reinterpret_cast<float(&)[2]>(vl));
        load_pair<2>(A.wu4, A.wu2, i, reinterpret_cast<float(&)[2]>(wuh), reinterpret_cast<float(&)[2]>(wul));
        load_pair<2>(A.wv4, A.wv2, i, reinterpret_cast<float(&)[2]>(wvh), reinterpret_cast<float(&)[2]>(wvl));
        const float2 aa = reinterpret_cast<const float2 *>(A.af)[i];
        const float2 wa = reinterpret_cast<const float2 *>(A.waf)[i];
        a[0] = __fadd_rn(aa.x, wa.x);
        a[1] = __fadd_rn(aa.y, wa.y);
    } else {
        load_pair<3>(A.u4, A.u2, i, uh, ul);
        load_pair<3>(A.v4, A.v2, i, vh, vl);
        load_pair<3>(A.wu4, A.wu2, i, wuh, wul);
        load_pair<3>(A.wv4, A.wv2, i, wvh, wvl);
        const float4 aa = reinterpret_cast<const float4 *>(A.af)[i];
        const float4 wa = reinterpret_cast<const float4 *>(A.waf)[i];
        a[0] = __fadd_rn(aa.x, wa.x);
        a[1] = __fadd_rn(aa.y, wa.y);
        a[2] = __fadd_rn(aa.z, wa.z);
    }
    const float dtf = (float)A.dt, hdt2f = (float)A.hdt2;
    for (int d = 0; d < A.dim; ++d) {
        df_add(uh[d], ul[d], wuh[d]);
        df_add(uh[d], ul[d], wul[d]);
        df_add(vh[d], vl[d], wvh[d]);
        df_add(vh[d], vl[d], wvl[d]);
    }
    float ph[3], pl[3];
    for (int d = 0; d < A.dim; ++d) {
        ph[d] = uh[d];
        pl[d] = ul[d];
        df_add(ph[d], pl[d], __fmaf_rn(dtf, vh[d], __fmaf_rn(dtf, vl[d], __fmul_rn(hdt2f, a[d]))));
    }
    if (A.dim == 2) {
        store_pair<2>(A.u4, A.u2, i, reinterpret_cast<float(&)[2]>(uh), reinterpret_cast<float(&)[2]>(ul));
        store_pair<2>(A.v4, A.v2, i, reinterpret_cast<float(&)[2]>(vh), reinterpret_cast<float(&)[2]>(vl));
        store_pair<2>(A.u4_pred, A.u2_pred, i, reinterpret_cast<float(&)[2]>(ph), reinterpret_cast<float(&)[2]>(pl));
        reinterpret_cast<float2 *>(A.af)[i] = make_float2(a[0], a[1]);
    } else {
        store_pair<3>(A.u4, A.u2, i, uh, ul);
        store_pair<3>(A.v4, A.v2, i, vh, vl);
        store_pair<3>(A.u4_pred, A.u2_pred, i, ph, pl);
        reinterpret_cast<float4 *>(A.af)[i] = make_float4(a[0], a[1], a[2], 0.f);
    }
}

// End of a coarse step in one pass: U_PD += W on the link segments (L), count
// the bits that changed in flagged words (a vs the step-start words b) into
// count[0], copy a into b (the next step's start words), copy lam into lam0.
__global__ void k_finish_step(const PDAddLink L, const int64_t nwords, const uint32_t *__restrict__ a,
                              uint32_t *__restrict__ b, const uint8_t *__restrict__ flag,
                              unsigned long long *count, const int64_t nlam, const double *__restrict__ lam,
                              double *__restrict__ lam0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L.seg_n[0] + L.seg_n[1])
        pd_add_link_node(L, i);
    unsigned c = 0;
    if (i < nwords) {
        const uint32_t ai = a[i], bi = b[i];
        if (flag[i] && ai != bi)
            c = __popc(ai ^ bi);
        if (ai != bi)
            b[i] = ai;
    }
    if (i < nlam)
        lam0[i] = lam[i];
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c)
        atomicAdd(count, (unsigned long long)c);
}

// ------------------------------------------------------------- launchers --
static inline unsigned grid_for_tiles(int64_t ntiles) { return (unsigned)((ntiles + 7) / 8); }

cudaError_t launch_pd_step_f64(int dim, const F64StepArgs &A, bool init, cudaStream_t s)
{
    if (A.fam.ntiles == 0)
        return cudaSuccess;
    const unsigned grid = grid_for_tiles(A.fam.ntiles);
    if (dim == 2)
        k_pd_step_f64<2><<<grid, 256, 0, s>>>(A, init ? 1 : 0);
    else
        k_pd_step_f64<3><<<grid, 256, 0, s>>>(A, init ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_pd_step_f32(int dim, const F32StepArgs &A, bool init, cudaStream_t s)
{
    if (A.fam.ntiles == 0)
        return cudaSuccess;
    const unsigned grid = grid_for_tiles(A.fam.ntiles);
    if (dim == 2)
        k_pd_step_f32<2><<<grid, 256, 0, s>>>(A, init ? 1 : 0);
    else
        k_pd_step_f32<3><<<grid, 256, 0, s>>>(A, init ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_pd_step_lattice2d(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    if (A.nx <= 0 || A.ny <= 0)
        return cudaSuccess;
    switch (A.tile) {
    case 0: return launch_lattice2d_t0(A, init, s);
    case 1: return launch_lattice2d_t1(A, init, s);
    case 2: return launch_lattice2d_t2(A, init, s);
    case 3: return launch_lattice2d_t3(A, init, s);
    case 4: return launch_lattice2d_t4(A, init, s);
    case 5: return launch_lattice2d_t5(A, init, s);
    case 6: return launch_lattice2d_t6(A, init, s);
    case 7: return launch_lattice2d_t7(A, init, s);
    case 8: return launch_lattice2d_t8(A, init, s);
    case 9: return launch_lattice2d_t9(A, init, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_damage_lattice(int64_t n, const uint32_t *mask, const uint32_t *exists, int words, double *phi,
                                  cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    k_damage_lattice<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, mask, exists, words, phi);
    return cudaGetLastError();
}

cudaError_t launch_damage(const SellView &fam, int packed, const double *V, double *phi, cudaStream_t s)
{
    if (fam.n == 0)
        return cudaSuccess;
    k_damage<<<(unsigned)((fam.n + 255) / 256), 256, 0, s>>>(fam, packed, V, phi);
    return cudaGetLastError();
}

cudaError_t launch_weighted_load(int dim, int64_t n, const double *b, const double *alpha64, const float *alpha32,
                                 double inv_h, double *wb64, float *wb32, unsigned long long *flag, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    k_weighted_load<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dim, n, b, alpha64, alpha32, inv_h, wb64, wb32,
                                                                 flag);
    return cudaGetLastError();
}

cudaError_t launch_interface_force(int dim, int64_t n, int64_t n_ov, const int32_t *ov_node, const int32_t *ov_k,
                                   const double *ov_N, int corners, const double *lam, int64_t nl, double inv_h,
                                   double *g64, float *g32, cudaStream_t s, double *g64b, float *g32b)
{
    if (n_ov == 0)
        return cudaSuccess;
    k_interface_force<<<(unsigned)((n_ov + 255) / 256), 256, 0, s>>>(dim, n, n_ov, ov_node, ov_k, ov_N, corners, lam,
                                                                      nl, inv_h, g64, g32, g64b, g32b);
    return cudaGetLastError();
}

cudaError_t launch_constraint(int dim, int64_t nl, const int64_t *gpd_ptr, const int32_t *gpd_col,
                              const double *gpd_val, int64_t npd, const double *v64, const float4 *v4,
                              const float2 *v2, double h, const int32_t *gfe_col, const double *gfe_val, int gfe_w,
                              int64_t nfe, const double *vfe, double sign_pd, double sign_fe, double *y,
                              cudaStream_t s, float2 *yf)
{
    const int64_t rows = (int64_t)dim * nl;
    if (rows == 0)
        return cudaSuccess;
    if (gfe_w > 32)
        return cudaErrorInvalidValue;
    k_constraint<<<(unsigned)((nl * 32 + 255) / 256), 256, 0, s>>>(dim, nl, gpd_ptr, gpd_col, gpd_val, npd, v64, v4,
                                                                      v2, h, gfe_col, gfe_val, gfe_w, nfe, vfe,
                                                                      sign_pd, sign_fe, y, 0, 0, yf);
    return cudaGetLastError();
}

cudaError_t launch_constraint_pd_many(int64_t nl, const int64_t *gpd_ptr, const int32_t *gpd_col,
                                      const double *gpd_val, int64_t npd, const float4 *v4, int64_t v4_stride,
                                      int nv, double h, double sign_pd, double *y, int64_t y_stride, cudaStream_t s)
{
    if (nl == 0 || nv <= 0)
        return cudaSuccess;
    if (nv > 65535)
        return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((nl * 32 + 255) / 256), (unsigned)nv);
    k_constraint<<<grid, 256, 0, s>>>(2, nl, gpd_ptr, gpd_col, gpd_val, npd, nullptr, v4, nullptr, h, nullptr, nullptr,
                                      0, 0, nullptr, sign_pd, 0.0, y, v4_stride, y_stride, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_finish_step(const PDAddLink &L, int64_t nwords, const uint32_t *a, uint32_t *b,
                               const uint8_t *word_flag, unsigned long long *count, int64_t nlam,
                               const double *lam, double *lam0, cudaStream_t s)
{
    const int64_t n =
        std::max<int64_t>(std::max<int64_t>(std::max<int64_t>(nwords, nlam), L.seg_n[0] + L.seg_n[1]), 1);
    k_finish_step<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, nwords, a, b, word_flag, count, nlam, lam,
                                                               lam0);
    return cudaGetLastError();
}

cudaError_t launch_unpack_f32(int dim, int64_t n, const float4 *p4, const float2 *p2, int accel, double h,
                              double *out, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    k_unpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dim, n, p4, p2, accel, h, out);
    return cudaGetLastError();
}

}  // namespace pdmts

// -------------------------------------------------- substep chains / graphs
// A chain of substeps alternates the two displacement buffers, so a captured
// graph of `len` substeps is keyed by the buffer parity it starts from (and by
// the interface-force schedule `sched` it bakes in). Graphs are dropped
// whenever a kernel argument or array changes.
using namespace pdmts;

int pd_invalidate_graphs(pdmts_pd *pd)
{
    for (auto &g : pd->graphs)
        if (g.exec)
            cudaGraphExecDestroy(g.exec);
    pd->graphs.clear();
    return PDMTS_OK;
}

// Launch one chain of `len` substeps with interface factors theta(k), either
// directly or by replaying its captured graph. Host bookkeeping (buffer
// parity, counters) is applied once per chain.
int pd_run_chain(pdmts_pd *pd, int len, int sched, const double *theta, cudaStream_t s, bool link)
{
    pdmts_ctx *ctx = pd->ctx;
    cudaEvent_t t0 = nullptr;
    if (!link)
        PDMTS_TRY(ctx->time_begin(&t0));
    int &cur = link ? pd->lk_cur : pd->cur;
    if (!pd->use_graphs || len < 2) {
        for (int k = 0; k < len; ++k) {
            pd->chain_follow = k > 0;
            pd->chain_k = k;
            const int r = pd->step(false, theta ? theta[k] : 0.0, s, link);
            pd->chain_follow = false;
            pd->chain_k = 0;
            PDMTS_TRY(r);
        }
        return link ? PDMTS_OK : ctx->time_end(t0, len);
    }
    const int p = cur + (link ? 2 : 0);
    cudaGraphExec_t exec = nullptr;
    for (auto &g : pd->graphs)
        if (g.parity == p && g.len == len && g.sched == sched)
            exec = g.exec;
    if (!exec) {
        const int cur0 = cur;
        const int64_t steps0 = pd->steps_done;
        const pdmts_stats st0 = ctx->stats;
        cudaGraph_t g = nullptr;
        PDMTS_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int r = PDMTS_OK;
        for (int k = 0; k < len && r == PDMTS_OK; ++k) {
            pd->chain_follow = k > 0;
            pd->chain_k = k;
            r = pd->step(false, theta ? theta[k] : 0.0, s, link);
        }
        pd->chain_follow = false;
        pd->chain_k = 0;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        cur = cur0;
        pd->steps_done = steps0;
        ctx->stats = st0;
        if (r != PDMTS_OK) {
            if (g)
                cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        pd->graphs.push_back({p, len, sched, exec});
    }
    PDMTS_CUDA_TRY(cudaGraphLaunch(exec, s));
    ctx->stats.graph_launches++;
    ctx->stats.kernel_launches += len;
    ctx->stats.pd_substeps += len;
    for (int k = 0; k < len; ++k)
        ctx->stats.bond_updates += pd->substep_bonds(link, k);
    if (!link)
        pd->steps_done += len;
    if (len & 1)
        cur = 1 - cur;
    return link ? PDMTS_OK : ctx->time_end(t0, len);
}

// nsteps plain substeps (theta = 0) in chains of `chunk`.
int pd_run_steps_graph(pdmts_pd *pd, int64_t nsteps, int chunk, cudaStream_t s)
{
    if (chunk < 1)
        chunk = 1;
    int64_t done = 0;
    while (nsteps - done >= chunk) {
        PDMTS_TRY(pd_run_chain(pd, chunk, 0, nullptr, s, false));
        done += chunk;
    }
    if (done < nsteps)
        PDMTS_TRY(pd_run_chain(pd, (int)(nsteps - done), 0, nullptr, s, false));
    return PDMTS_OK;
}
