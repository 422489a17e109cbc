// lattice2d.cuh -- the FP32-bulk PD substep on a regular 2D lattice
// (arXiv 2403.03605, Eq. 1-4 with the Arlequin bond weights of Sec. 3.2 and
// the per-node update of Eq. 38). Each tile configuration (strip height KR,
// resident CTAs per SM) is instantiated in a translation unit of its own.
#pragma once

#include <algorithm>
#include <utility>
#include <type_traits>

#include "f32_device.cuh"

namespace pdmts {

// ---------------------------------------------------------- 2D lattice ----
// A CTA owns a 32 x (8 KR) node tile of the nx * ny lattice and each thread a
// column strip of KR nodes. The displacement halo ((32 + 6) x (8 KR + 6)
// nodes) is staged once in shared memory. Bonds are visited column by column
// of the stencil (dx = -3..3, top to bottom): a thread reads each halo value of
// a column once and applies it to every node of its strip within reach, so a
// strip reads 7 KR + 22 values for its 28 KR bonds. The family is implicit
// (offset k of the 28-offset stencil); per node only its bond word is read.
//
// Bond (i, j) with lattice offset d and eta = u_j - u_i (compensated pairs):
//   p = 2 d.eta / |d|^2,  q = p + |eta|^2 / |d|^2 = (|d + eta|^2 - |d|^2) / |d|^2
//   breaks when q >= s0 (2 + s0)                         (Eq. 3-4, squared)
//   linear force (coef |d|^2 / 2) p d = coef (d.eta) d   (Eq. 2)
//   PMB force coef |d|^4 q / ((|d + eta| + |d|) |d + eta|) (d + eta)
// Every expression is even or odd under (d, eta) -> (-d, -eta), so the two
// directions of a bond reach the same decision and opposite forces.
namespace lat2d {
constexpr int HX = TX + 2 * R;
// reach of stencil column dx: |dy| <= RY(dx) with dx^2 + dy^2 <= 9
__host__ __device__ constexpr int RY(int dx) { return dx == 0 ? 3 : (dx >= -2 && dx <= 2) ? 2 : 0; }
__host__ __device__ constexpr int KOF(int dx, int dy)
{
    for (int k = 0; k < NS; ++k)
        if (DX(k) == dx && DY(k) == dy)
            return k;
    return -1;
}
}  // namespace lat2d

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// f(E - 1), f(E - 2), ..., f(B)
template <int B, int E, class F>
__device__ __forceinline__ void static_for_desc(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, E - 1>{});
        static_for_desc<B, E - 1>(f);
    }
}

// Canonical bond order of a node. Every path (pair, warp fast path, masked)
// sums a node's bond forces in this order, so every path and every tile
// configuration gives the same bits: first the 14 bonds d of the half stencil
// H+ = {dx > 0} + {dx = 0, dy > 0}, by column dx = 0..3 and dy ascending
// (PDX/PDY below); then the 14 bonds -d, d in H+, in the same order of d.
namespace lat2d {
constexpr int NP = 14;
__host__ __device__ constexpr int PDX(int k)
{
    constexpr int t[NP] = {0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3};
    return t[k];
}
__host__ __device__ constexpr int PDY(int k)
{
    constexpr int t[NP] = {1, 2, 3, -2, -1, 0, 1, 2, -2, -1, 0, 1, 2, 0};
    return t[k];
}
__host__ __device__ constexpr int KP(int dx, int dy)
{
    for (int k = 0; k < NP; ++k)
        if (PDX(k) == dx && PDY(k) == dy)
            return k;
    return -1;
}
// rows of column dx that hold H+ bonds: dy in [PLO(dx), RY(dx)]
__host__ __device__ constexpr int PLO(int dx) { return dx == 0 ? 1 : -RY(dx); }
}  // namespace lat2d

// Bond word of a node with all 28 bonds present and intact.
constexpr uint32_t kFullWord = (1u << lat2d::NS) - 1u;

// acc += s * D for a compile-time integer D, rounded once like fma(s, D, acc)
template <int D>
__device__ __forceinline__ void lattice_acc(float &acc, const float s)
{
    if constexpr (D == 1)
        acc = __fadd_rn(acc, s);
    else if constexpr (D == -1)
        acc = __fsub_rn(acc, s);
    else if constexpr (D != 0)
        acc = __fmaf_rn(s, (float)D, acc);
}

// One bond of the node with state nu = -u_i (and weight ai); accumulates its
// force into f and returns the scalar s of the linear law's f = s d.
template <int DX, int DY, bool ALPHA, bool PMB, bool MASKED>
__device__ __forceinline__ float lattice_bond(const float4 uj, const float aj, const float4 nu, const float ai,
                                              const Lat2DArgs &A, const uint32_t m0, uint32_t &m, float2 &f,
                                              float &qmax)
{
    constexpr int r2 = DX * DX + DY * DY;
    constexpr int K = lat2d::KOF(DX, DY);
    static_assert(K >= 0, "offset outside the stencil");
    constexpr float ir2 = 1.f / (float)r2;
    constexpr float cx = 2.f * (float)DX / (float)r2, cy = 2.f * (float)DY / (float)r2;
    const float2 eh = __fadd2_rn(make_float2(uj.x, uj.y), make_float2(nu.x, nu.y));
    const float2 el = __fadd2_rn(make_float2(uj.z, uj.w), make_float2(nu.z, nu.w));
    const float2 eta = __fadd2_rn(eh, el);
    float p;
    if constexpr (DY == 0)
        p = __fmul_rn(cx, eta.x);
    else if constexpr (DX == 0)
        p = __fmul_rn(cy, eta.y);
    else
        p = __fmaf_rn(cy, eta.y, __fmul_rn(cx, eta.x));
    const float e2 = __fmaf_rn(eta.y, eta.y, __fmul_rn(eta.x, eta.x));
    const float q = __fmaf_rn(e2, ir2, p);
    float c = PMB ? A.cpmb[r2] : A.clin[r2];
    if constexpr (ALPHA)
        c = __fmul_rn(c, bond_weight(ai, aj));
    float sc;
    float2 dir = make_float2(0.f, 0.f);
    if constexpr (!PMB) {
        sc = __fmul_rn(c, p);
    } else {
        constexpr float rd = r2 == 1 ? 1.f : r2 == 2 ? 1.41421354f : r2 == 4 ? 2.f : r2 == 5 ? 2.23606801f
                             : r2 == 8 ? 2.82842708f : 3.f;
        const float ry = __fmul_rn(rd, __fsqrt_rn(fmaxf(__fadd_rn(1.f, q), 0.f)));
        sc = __fdiv_rn(__fmul_rn(c, q), __fmul_rn(__fadd_rn(ry, rd), ry));
        dir = __fadd2_rn(make_float2((float)DX, (float)DY), eta);
    }
    float s = sc;
    if constexpr (!MASKED) {
        qmax = fmaxf(qmax, q);
    } else {
        const bool on = (m0 >> K) & 1u;
        const bool brk = on && A.nd.breaking && q >= A.qthr;
        if (brk)
            m &= ~(1u << K);
        s = (on && !brk) ? sc : 0.f;
    }
    if constexpr (!PMB) {
        // f += s d with the integer offset as an immediate (a constant vector
        // operand would hold registers); identical rounding to fma(s, d, f)
        lattice_acc<DX>(f.x, s);
        lattice_acc<DY>(f.y, s);
    } else {
        f = __ffma2_rn(make_float2(s, s), dir, f);
    }
    return s;
}

// All 28 bonds of the KR nodes of one strip with every bond taken as intact
// (fast path), in the canonical order: the H+ columns dx = 0..3 with rows
// ascending, then the H- columns dx = 0, -1, -2, -3 with rows descending. A
// thread reads each halo value of a column once and applies it to every node
// of its strip within reach; qmax collects the largest q.
template <int KR, bool ALPHA, bool PMB>
__device__ __forceinline__ void lattice_strip(const float4 (*su)[lat2d::HX], const float (*sal)[lat2d::HX],
                                              const int hy0, const int hx0, const Lat2DArgs &A,
                                              const float4 (&nu)[KR], const float (&ai)[KR],
                                              const uint32_t (&m0)[KR], uint32_t (&m)[KR], float2 (&f)[KR],
                                              float (&qmax)[KR])
{
    using namespace lat2d;
    static_for<0, R + 1>([&](auto dxc) {
        constexpr int dx = decltype(dxc)::value;
        constexpr int ry = RY(dx), lo = PLO(dx);
        // keep the shared-memory reads of one column together: bounds how far
        // the scheduler hoists loads, and with it the live registers
        asm volatile("" ::: "memory");
        static_for<lo, KR + ry>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const float4 uj = su[hy0 + j][hx0 + dx];
            const float aj = ALPHA ? sal[hy0 + j][hx0 + dx] : 0.f;
            static_for<0, KR>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr int dy = j - r;
                if constexpr (dy >= lo && dy <= ry)
                    lattice_bond<dx, dy, ALPHA, PMB, false>(uj, aj, nu[r], ai[r], A, m0[r], m[r], f[r], qmax[r]);
            });
        });
    });
    static_for<0, R + 1>([&](auto c) {
        constexpr int dx = -decltype(c)::value;
        constexpr int ry = RY(dx), hi = -PLO(-dx);  // H- rows of column dx: dy in [-ry, hi]
        asm volatile("" ::: "memory");
        static_for_desc<-ry, KR + hi>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const float4 uj = su[hy0 + j][hx0 + dx];
            const float aj = ALPHA ? sal[hy0 + j][hx0 + dx] : 0.f;
            static_for<0, KR>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr int dy = j - r;
                if constexpr (dy >= -ry && dy <= hi)
                    lattice_bond<dx, dy, ALPHA, PMB, false>(uj, aj, nu[r], ai[r], A, m0[r], m[r], f[r], qmax[r]);
            });
        });
    });
}

// The 28 bonds of one node with its bond bits: exact breaking, absent bonds
// skipped, in the canonical order (H+ by offset index, then -d for d in H+),
// so a warp that takes this path without a break gets the fast path's bits.
template <bool ALPHA, bool PMB>
__device__ __forceinline__ void lattice_node_masked(const float4 (*su)[lat2d::HX], const float (*sal)[lat2d::HX],
                                                    const int hy, const int hx, const Lat2DArgs &A, const float4 nu,
                                                    const float ai, const uint32_t m0, uint32_t &m, float2 &f)
{
    using namespace lat2d;
    static_for<0, 2>([&](auto sc) {
        constexpr int sg = decltype(sc)::value ? -1 : 1;
        static_for<0, NP>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int dx = sg * PDX(k), dy = sg * PDY(k);
            const float4 uj = su[hy + dy][hx + dx];
            const float aj = ALPHA ? sal[hy + dy][hx + dx] : 0.f;
            float qunused = 0.f;
            lattice_bond<dx, dy, ALPHA, PMB, true>(uj, aj, nu, ai, A, m0, m, f, qunused);
        });
    });
}

// The masked path over a strip: a rolled loop over its nodes (the rare path
// near cracks and edges; one copy of the bond code, one node's state live).
template <int KR, bool ALPHA, bool PMB>
__device__ __forceinline__ void lattice_strip_masked(const float4 (*su)[lat2d::HX], const float (*sal)[lat2d::HX],
                                                     const int hy0, const int hx0, const Lat2DArgs &A,
                                                     const float4 (&nu)[KR], const float (&ai)[KR],
                                                     const uint32_t (&m0)[KR], uint32_t (&m)[KR], float2 (&f)[KR])
{
#pragma unroll 1
    for (int r = 0; r < KR; ++r) {
        float4 nur = nu[0];
        float air = ai[0];
        uint32_t m0r = m0[0];
        static_for<1, KR>([&](auto rc) {
            constexpr int q = decltype(rc)::value;
            if (r == q) {
                nur = nu[q];
                air = ai[q];
                m0r = m0[q];
            }
        });
        uint32_t mr = m0r;
        float2 fr = make_float2(0.f, 0.f);
        lattice_node_masked<ALPHA, PMB>(su, sal, hy0 + r, hx0, A, nur, air, m0r, mr, fr);
        static_for<0, KR>([&](auto rc) {
            constexpr int q = decltype(rc)::value;
            if (r == q) {
                m[q] = mr;
                f[q] = fr;
            }
        });
    }
}

// ------------------------------------------------------- tile staging ----
// Every input of a tile is staged in shared memory with asynchronous copies
// (cp.async, zero-filled outside the lattice) in two groups:
//   A: the displacement halo (and weight halo), row by row, and the bond
//      words of each thread's own strip: needed before the bonds;
//   B: v, a, 1/m and the loads of each thread's own strip: needed only by the
//      per-node update after the bonds, so their latency hides behind them.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, const bool pred)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, const bool pred)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, const bool pred)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Inputs of one tile in shared memory.
template <int KR>
struct LatStage {
    static constexpr int TYK = lat2d::TY * KR, HY = TYK + 2 * lat2d::R;
    alignas(16) float4 u[HY][lat2d::HX];
    alignas(16) float4 v[TYK][lat2d::TX];
    alignas(16) float2 a[TYK][lat2d::TX];
    alignas(16) float al[HY][lat2d::HX];
    alignas(16) float im[TYK][lat2d::TX];
    alignas(16) uint32_t mk[TYK][lat2d::TX];
    alignas(16) float wb[2][TYK][lat2d::TX];
    alignas(16) float g[2][TYK][lat2d::TX];
};

template <int KR>
__device__ __forceinline__ void lattice_issue_a(LatStage<KR> &S, const Lat2DArgs &A, const int x0, const int y0)
{
    using namespace lat2d;
    constexpr int HY = LatStage<KR>::HY;
    const int nx = A.nx, ny = A.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int hy = warp; hy < HY; hy += 8) {
        const int gy = y0 + hy - R;
        const bool row_in = gy >= 0 && gy < ny;
        for (int hx = lane; hx < HX; hx += 32) {
            const int gx = x0 + hx - R;
            const bool in = row_in && gx >= 0 && gx < nx;
            const int64_t gi = in ? (int64_t)gy * nx + gx : 0;
            cp_async16(&S.u[hy][hx], A.nd.u4_in + gi, in);
            if (A.alpha)
                cp_async4(&S.al[hy][hx], A.alpha + gi, in);
        }
    }
    const int x = x0 + lane;
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        const int y = y0 + warp * KR + r;
        const bool in = x < nx && y < ny;
        cp_async4(&S.mk[warp * KR + r][lane], A.mask + (in ? (int64_t)y * nx + x : 0), in);
    }
}

template <int KR>
__device__ __forceinline__ void lattice_issue_b(LatStage<KR> &S, const Lat2DArgs &A, const int x0, const int y0)
{
    const F32NodeArgs &N = A.nd;
    const int nx = A.nx, ny = A.ny;
    const int64_t n = N.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float2 *a2 = reinterpret_cast<const float2 *>(N.a);
    const int x = x0 + lane;
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        const int ry = warp * KR + r, y = y0 + ry;
        const bool in = x < nx && y < ny;
        const int64_t i = in ? (int64_t)y * nx + x : 0;
        cp_async16(&S.v[ry][lane], N.v4 + i, in);
        cp_async8(&S.a[ry][lane], a2 + i, in);
        cp_async4(&S.im[ry][lane], N.inv_m + i, in);
        if (N.wb) {
            cp_async4(&S.wb[0][ry][lane], N.wb + i, in);
            cp_async4(&S.wb[1][ry][lane], N.wb + (in ? n + i : 0), in);
        }
        if (N.g) {
            cp_async4(&S.g[0][ry][lane], N.g + i, in);
            cp_async4(&S.g[1][ry][lane], N.g + (in ? n + i : 0), in);
        }
    }
}

// The substep of the tile at (x0, y0) from its staged inputs. On entry this
// thread's group A has landed; group B is awaited with cp.async.wait_group
// WAIT_B before the per-node update. Returns the bonds this thread broke.
template <bool PMB, int KR, int WAIT_B>
__device__ __forceinline__ unsigned lattice_tile(LatStage<KR> &S, const Lat2DArgs &A, const int x0, const int y0,
                                                 const int init)
{
    using namespace lat2d;
    constexpr int HY = LatStage<KR>::HY;
    const F32NodeArgs &N = A.nd;
    const int nx = A.nx, ny = A.ny;
    bool any_alpha = false;
    if (A.alpha)
        for (int q = threadIdx.x; q < HY * HX; q += blockDim.x)
            any_alpha |= (&S.al[0][0])[q] != 0.f;
    // a tile whose halo carries no Arlequin weight evaluates every bond with
    // weight 1 exactly, so it can skip the weights (the barrier also makes
    // every thread's group A visible)
    const bool has_alpha = __syncthreads_or(any_alpha) != 0;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int hx0 = tx + R, hy0 = ty * KR + R;
    const int x = x0 + tx, ys = y0 + ty * KR;  // the strip: nodes (x, ys + r), r < KR
    float4 nu[KR];
    float ai[KR], qmax[KR];
    uint32_t m0[KR], m[KR];
    float2 f[KR];
    unsigned vbits = 0;  // bit r: node r of the strip lies in the lattice
    bool full = true;
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        const bool valid = x < nx && ys + r < ny;
        vbits |= valid ? 1u << r : 0u;
        m0[r] = valid ? S.mk[ty * KR + r][tx] : 0u;
        m[r] = m0[r];
        full = full && (m0[r] == kFullWord || !valid);
        const float4 u = S.u[hy0 + r][hx0];
        nu[r] = make_float4(-u.x, -u.y, -u.z, -u.w);
        ai[r] = has_alpha ? S.al[hy0 + r][hx0] : 0.f;
        f[r] = make_float2(0.f, 0.f);
        qmax[r] = -INFINITY;
    }
    // Fast path: every node of the warp has all bonds intact; evaluate all
    // bonds without per-bond control flow and only note the largest q. If a
    // bond reached the critical stretch (rare), redo the warp bond by bond.
    bool fast = __all_sync(0xffffffffu, full);
    if (fast) {
        if (has_alpha)
            lattice_strip<KR, true, PMB>(S.u, S.al, hy0, hx0, A, nu, ai, m0, m, f, qmax);
        else
            lattice_strip<KR, false, PMB>(S.u, S.al, hy0, hx0, A, nu, ai, m0, m, f, qmax);
        bool hit = false;
#pragma unroll
        for (int r = 0; r < KR; ++r)
            hit = hit || (((vbits >> r) & 1u) && qmax[r] >= A.qthr);
        if (N.breaking && __any_sync(0xffffffffu, hit))
            fast = false;
    }
    if (!fast) {
        if (has_alpha)
            lattice_strip_masked<KR, true, PMB>(S.u, S.al, hy0, hx0, A, nu, ai, m0, m, f);
        else
            lattice_strip_masked<KR, false, PMB>(S.u, S.al, hy0, hx0, A, nu, ai, m0, m, f);
    }
    cp_async_wait<WAIT_B>();  // this thread's group B (its own strip) has landed
    unsigned nbroken = 0;
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        if (!((vbits >> r) & 1u))
            continue;
        const int64_t i = (int64_t)(ys + r) * nx + x;
        if (m[r] != m0[r]) {
            A.mask[i] = m[r];
            nbroken += __popc(m0[r] ^ m[r]);
        }
        const int ry = ty * KR + r;
        const float fr[2] = {f[r].x, f[r].y};
        float uh[2] = {-nu[r].x, -nu[r].y}, ul[2] = {-nu[r].z, -nu[r].w};
        const float2 wb = N.wb ? make_float2(S.wb[0][ry][tx], S.wb[1][ry][tx]) : make_float2(0.f, 0.f);
        const float2 g = N.g ? make_float2(S.g[0][ry][tx], S.g[1][ry][tx]) : make_float2(0.f, 0.f);
        finish_node_2d_vals(N, i, fr, uh, ul, S.a[ry][tx], S.v[ry][tx], S.im[ry][tx], wb, g, init);
    }
    return nbroken;
}

// Tile row of tile-list row `by`: all tile rows, or the rows of up to two
// windows [win_lo, win_lo + win_n).
__device__ __forceinline__ int lattice_trow(const Lat2DArgs &A, const int by)
{
    return A.win_n[0] > 0 ? (by < A.win_n[0] ? A.win_lo[0] + by : A.win_lo[1] + by - A.win_n[0]) : by;
}

// Programmatic dependent launch inside a substep chain: the CTAs of substep
// k + 1 may be scheduled while substep k drains; every global access (the
// ping-pong u buffers, v, a and the bond words are all read and written)
// waits for substep k to complete. Outside such a launch both are no-ops.
__device__ __forceinline__ void lattice_chain_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One CTA per tile (grid: tile columns x tile rows).
template <bool PMB, int KR, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pd_step_lattice2d(const Lat2DArgs A, const int init)
{
    extern __shared__ __align__(16) unsigned char lat_smem[];
    LatStage<KR> &S = *reinterpret_cast<LatStage<KR> *>(lat_smem);
    const int x0 = blockIdx.x * lat2d::TX, y0 = lattice_trow(A, (int)blockIdx.y) * LatStage<KR>::TYK;
    lattice_chain_entry();
    lattice_issue_a<KR>(S, A, x0, y0);
    cp_async_commit();
    lattice_issue_b<KR>(S, A, x0, y0);
    cp_async_commit();
    cp_async_wait<1>();
    const unsigned nbroken = lattice_tile<PMB, KR, 0>(S, A, x0, y0, init);
    count_broken(A.nd.broken, nbroken);
}

// Persistent variant: a grid of (SMs x resident CTAs) walks the tile list in
// order, each CTA staging its next tile while it computes the current one
// (two stages). The same per-tile code, so the same bits.
template <bool PMB, int KR, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pd_step_lattice2d_pipe(const Lat2DArgs A, const int init,
                                                                       const int ntiles)
{
    constexpr int TYK = LatStage<KR>::TYK;
    extern __shared__ __align__(16) unsigned char lat_smem[];
    LatStage<KR> *stages = reinterpret_cast<LatStage<KR> *>(lat_smem);
    const int ntx = (A.nx + lat2d::TX - 1) / lat2d::TX;
    const int G = gridDim.x;
    auto issue = [&](LatStage<KR> &S, const int t) {
        if (t < ntiles) {
            const int x0 = (t % ntx) * lat2d::TX, y0 = lattice_trow(A, t / ntx) * TYK;
            lattice_issue_a<KR>(S, A, x0, y0);
            cp_async_commit();
            lattice_issue_b<KR>(S, A, x0, y0);
            cp_async_commit();
        } else {  // empty groups keep the group count uniform
            cp_async_commit();
            cp_async_commit();
        }
    };
    lattice_chain_entry();
    issue(stages[0], blockIdx.x);
    issue(stages[1], blockIdx.x + G);
    unsigned nbroken = 0;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++k) {
        LatStage<KR> &S = stages[k & 1];
        // pending, newest first: B(t+G), A(t+G), B(t); A(t) has landed
        cp_async_wait<3>();
        const int x0 = (t % ntx) * lat2d::TX, y0 = lattice_trow(A, t / ntx) * TYK;
        nbroken += lattice_tile<PMB, KR, 2>(S, A, x0, y0, init);
        __syncthreads();  // every thread is done with S
        issue(S, t + 2 * G);
    }
    cp_async_wait<0>();
    count_broken(A.nd.broken, nbroken);
}

// Batched substep over several lattices: one CTA per work item (instance,
// tile in that instance's tile list); the CTA copies its instance's arguments
// to shared memory once. The per-tile code is the single-lattice one, so a
// batched substep gives every instance the bits of its own substep.
template <bool PMB, int KR, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pd_step_lattice2d_batch(const Lat2DArgs *__restrict__ args,
                                                                        const int2 *__restrict__ work,
                                                                        const int init)
{
    __shared__ __align__(16) Lat2DArgs sA;
    extern __shared__ __align__(16) unsigned char lat_smem[];
    LatStage<KR> &S = *reinterpret_cast<LatStage<KR> *>(lat_smem);
    const int2 w = work[blockIdx.x];
    static_assert(sizeof(Lat2DArgs) % 4 == 0, "argument block copied as words");
    const int *src = reinterpret_cast<const int *>(args + w.x);
    int *dst = reinterpret_cast<int *>(&sA);
    for (int q = threadIdx.x; q < (int)(sizeof(Lat2DArgs) / 4); q += blockDim.x)
        dst[q] = src[q];
    __syncthreads();
    const Lat2DArgs &A = sA;
    const int ntx = (A.nx + lat2d::TX - 1) / lat2d::TX;
    const int x0 = (w.y % ntx) * lat2d::TX, y0 = lattice_trow(A, w.y / ntx) * LatStage<KR>::TYK;
    lattice_issue_a<KR>(S, A, x0, y0);
    cp_async_commit();
    lattice_issue_b<KR>(S, A, x0, y0);
    cp_async_commit();
    cp_async_wait<1>();
    const unsigned nbroken = lattice_tile<PMB, KR, 0>(S, A, x0, y0, init);
    count_broken(A.nd.broken, nbroken);
}

// Tile rows of the launch (all, or the windows converted to this tile height).
template <int TYK>
__host__ int lattice_tile_rows(Lat2DArgs &A, const Lat2DArgs &A0)
{
    int rows = (A0.ny + TYK - 1) / TYK;
    if (A0.win_n[0] > 0) {
        // windows of TY-row units to tile rows of this tile height (merged when they touch)
        int lo[2] = {0, 0}, cnt[2] = {0, 0}, nw = 0;
        for (int w = 0; w < 2; ++w) {
            if (A0.win_n[w] <= 0)
                continue;
            const int t0 = A0.win_lo[w] * lat2d::TY / TYK;
            const int r1 = std::min(A0.ny, (A0.win_lo[w] + A0.win_n[w]) * lat2d::TY);
            const int t1 = std::max(t0 + 1, (r1 + TYK - 1) / TYK);
            if (nw > 0 && t0 <= lo[nw - 1] + cnt[nw - 1]) {
                cnt[nw - 1] = std::max(cnt[nw - 1], t1 - lo[nw - 1]);
            } else {
                lo[nw] = t0;
                cnt[nw] = t1 - t0;
                ++nw;
            }
        }
        for (int w = 0; w < 2; ++w) {
            A.win_lo[w] = lo[w];
            A.win_n[w] = cnt[w];
        }
        rows = cnt[0] + cnt[1];
    }
    return rows;
}

// One-time set-up of a kernel: opt in to its dynamic shared memory and read
// how many CTAs an SM holds (host calls only, no stream work).
template <class K>
cudaError_t lattice_prepare(K kern, size_t smem, int &ctas)
{
    if (ctas > 0)
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
    if (e != cudaSuccess)
        return e;
    if (nb < 1)
        return cudaErrorInvalidConfiguration;
    ctas = nb;
    return cudaSuccess;
}

// Launch with 256 threads; `pdl` adds the programmatic-serialisation
// attribute (the kernel begins with lattice_chain_entry).
template <typename... P, typename... Q>
cudaError_t lattice_launch(void (*kern)(P...), const dim3 grid, const size_t smem, cudaStream_t s, const bool pdl,
                           Q &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Q>(args)...);
}

template <int KR, int MINB>
cudaError_t launch_lattice_pipe(const Lat2DArgs &A0, bool init, cudaStream_t s)
{
    constexpr size_t smem = 2 * sizeof(LatStage<KR>);
    static int ctas[2] = {0, 0};
    const auto kern = A0.nd.pmb ? k_pd_step_lattice2d_pipe<true, KR, MINB> : k_pd_step_lattice2d_pipe<false, KR, MINB>;
    int &nb = ctas[A0.nd.pmb ? 1 : 0];
    cudaError_t e = lattice_prepare(kern, smem, nb);
    if (e != cudaSuccess)
        return e;
    Lat2DArgs A = A0;
    const int rows = lattice_tile_rows<LatStage<KR>::TYK>(A, A0);
    const int ntiles = ((A.nx + lat2d::TX - 1) / lat2d::TX) * rows;
    const int grid = std::max(1, std::min(ntiles, A.num_sms * nb));
    return lattice_launch(kern, dim3((unsigned)grid), smem, s, A.pdl != 0, A, init ? 1 : 0, ntiles);
}

template <int KR, int MINB>
cudaError_t launch_lattice_kr(const Lat2DArgs &A0, bool init, cudaStream_t s)
{
    constexpr size_t smem = sizeof(LatStage<KR>);
    static int ctas[2] = {0, 0};
    const auto kern = A0.nd.pmb ? k_pd_step_lattice2d<true, KR, MINB> : k_pd_step_lattice2d<false, KR, MINB>;
    cudaError_t e = lattice_prepare(kern, smem, ctas[A0.nd.pmb ? 1 : 0]);
    if (e != cudaSuccess)
        return e;
    Lat2DArgs A = A0;
    const unsigned rows = (unsigned)lattice_tile_rows<LatStage<KR>::TYK>(A, A0);
    const dim3 grid((unsigned)((A.nx + lat2d::TX - 1) / lat2d::TX), rows);
    return lattice_launch(kern, grid, smem, s, A.pdl != 0, A, init ? 1 : 0);
}

template <int KR, int MINB>
int lattice_batch_prepare(Lat2DArgs &A)
{
    const Lat2DArgs A0 = A;
    const int rows = lattice_tile_rows<LatStage<KR>::TYK>(A, A0);
    return ((A.nx + lat2d::TX - 1) / lat2d::TX) * rows;
}

template <int KR, int MINB>
cudaError_t launch_lattice_batch(const Lat2DArgs *d_args, const int2 *d_work, int nwork, bool pmb, cudaStream_t s)
{
    if (nwork <= 0)
        return cudaSuccess;
    constexpr size_t smem = sizeof(LatStage<KR>);
    static int ctas[2] = {0, 0};
    const auto kern = pmb ? k_pd_step_lattice2d_batch<true, KR, MINB> : k_pd_step_lattice2d_batch<false, KR, MINB>;
    cudaError_t e = lattice_prepare(kern, smem, ctas[pmb ? 1 : 0]);
    if (e != cudaSuccess)
        return e;
    kern<<<nwork, 256, smem, s>>>(d_args, d_work, 0);
    return cudaGetLastError();
}

}  // namespace pdmts
