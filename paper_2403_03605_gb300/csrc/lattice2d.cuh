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
// the weight halo is staged from column x0 - R - 1 (16-byte aligned for the
// tensor copy), so its rows are HX + 2 wide and column hx sits at hx + 1
constexpr int HXA = HX + 2;
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

// Watch of the fast path for bonds at or past the critical stretch: w.x is
// the largest p (linear law) or q (PMB) of the bonds seen, w.y the largest
// |eta| component (linear law; 0 for PMB). Every bond has
// q = p + |eta|^2 / |d|^2 <= p + 2 max(|eta_x|, |eta_y|)^2, so when the bound
// w.x + 2 w.y^2 of a strip stays below qfast = qthr (1 - 2^-12) none of its
// bonds reached qthr (the margin covers the rounding of q and of the bound)
// and the masked path, which decides each bond exactly, would break nothing.
__device__ __forceinline__ float watch_bound(const float2 w) { return __fmaf_rn(2.f * w.y, w.y, w.x); }
constexpr float2 kWatch0 = {-INFINITY, 0.f};

// One bond of the node with state nu = -u_i (and weight ai); accumulates its
// force into f and returns the scalar s of the linear law's f = s d.
template <int DX, int DY, bool ALPHA, bool PMB, bool MASKED>
__device__ __forceinline__ float lattice_bond(const float4 uj, const float aj, const float4 nu, const float ai,
                                              const Lat2DArgs &A, const uint32_t m0, uint32_t &m, float2 &f,
                                              float2 &watch)
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
        if constexpr (PMB) {
            watch.x = fmaxf(watch.x, q);
        } else {
            watch.x = fmaxf(watch.x, p);
            watch.y = fmaxf(watch.y, fmaxf(fabsf(eta.x), fabsf(eta.y)));
        }
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
// of its strip within reach; watch collects the break watch of each node.
template <int KR, bool ALPHA, bool PMB>
__device__ __forceinline__ void lattice_strip(const float4 (*su)[lat2d::HX], const float (*sal)[lat2d::HXA],
                                              const int hy0, const int hx0, const Lat2DArgs &A,
                                              const float4 (&nu)[KR], const float (&ai)[KR],
                                              const uint32_t (&m0)[KR], uint32_t (&m)[KR], float2 (&f)[KR],
                                              float2 (&watch)[KR])
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
                    lattice_bond<dx, dy, ALPHA, PMB, false>(uj, aj, nu[r], ai[r], A, m0[r], m[r], f[r], watch[r]);
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
                    lattice_bond<dx, dy, ALPHA, PMB, false>(uj, aj, nu[r], ai[r], A, m0[r], m[r], f[r], watch[r]);
            });
        });
    });
}

// The 28 bonds of one node with its bond bits: exact breaking, absent bonds
// skipped, in the canonical order (H+ by offset index, then -d for d in H+),
// so a warp that takes this path without a break gets the fast path's bits.
template <bool ALPHA, bool PMB>
__device__ __forceinline__ void lattice_node_masked(const float4 (*su)[lat2d::HX], const float (*sal)[lat2d::HXA],
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
            float2 wunused = kWatch0;
            lattice_bond<dx, dy, ALPHA, PMB, true>(uj, aj, nu, ai, A, m0, m, f, wunused);
        });
    });
}

// The masked path over a strip: a rolled loop over its nodes (the rare path
// near cracks and edges; one copy of the bond code, one node's state live).
template <int KR, bool ALPHA, bool PMB>
__device__ __forceinline__ void lattice_strip_masked(const float4 (*su)[lat2d::HX], const float (*sal)[lat2d::HXA],
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

// ---------------------------------------------------- tensor-copy staging ----
// The same two groups as tensor copies (cp.async.bulk.tensor) issued by one
// thread, each completing on an mbarrier. Out-of-lattice parts of a box read
// as zeros, like the predicated copies above. Every wait is bounded: after
// kTmaPolls polls (each suspends for at most ~1 us; a tile's first wait takes
// its limit from Lat2DArgs::first_polls, which only tests lower) it gives up;
// the CTA then raises counter word [2] (reported by the host as
// PDMTS_ERR_TIMEOUT), waits once more with the full limit for its copies and
// returns without touching global memory. The substep's result is then
// undefined.
constexpr unsigned kTmaPolls = kWaitPolls;

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, const unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, const unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, const unsigned parity, const unsigned polls = kTmaPolls)
{
    for (unsigned k = 0; k < polls; ++k) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (done)
            return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, const int c0, const int c1,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, const int c0, const int c1,
                                            const int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}],"
        " [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_gave_up(const Lat2DArgs &A)
{
    if (threadIdx.x == 0 && A.nd.broken)
        atomicOr(A.nd.broken + 2, 1ull);
}

// Inputs of one tile in shared memory.
template <int KR>
struct LatStage {
    static constexpr int TYK = lat2d::TY * KR, HY = TYK + 2 * lat2d::R;
    alignas(128) float4 u[HY][lat2d::HX];
    alignas(128) float4 v[TYK][lat2d::TX];
    alignas(128) float2 a[TYK][lat2d::TX];
    alignas(128) float al[HY][lat2d::HXA];
    alignas(128) float im[TYK][lat2d::TX];
    alignas(128) uint32_t mk[TYK][lat2d::TX];
    alignas(128) float wb[2][TYK][lat2d::TX];
    alignas(128) float g[2][TYK][lat2d::TX];
    alignas(8) uint64_t bar[2];  // tensor-copy barriers of groups A and B
    // the weight halo indexed like u: alh()[hy][hx]
    __device__ const float (*alh() const)[lat2d::HXA]
    {
        return reinterpret_cast<const float(*)[lat2d::HXA]>(&al[0][1]);
    }
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
                cp_async4(&S.al[hy][hx + 1], A.alpha + gi, in);
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

// Both groups of a tile as tensor copies (thread 0 only); box bytes equal
// the stage arrays' sizes, so each barrier completes when its group landed.
template <int KR>
__device__ __forceinline__ void lattice_tma_issue(LatStage<KR> &S, const LatMaps &M, const Lat2DArgs &A,
                                                  const int x0, const int y0)
{
    using namespace lat2d;
    const bool al = A.alpha != nullptr, wb = A.nd.wb != nullptr, g = A.nd.g != nullptr;
    mbar_expect_tx(&S.bar[0], (unsigned)(sizeof(S.u) + (al ? sizeof(S.al) : 0) + sizeof(S.mk)));
    tma_load_3d(&S.u[0][0], &M.u, 0, x0 - R, y0 - R, &S.bar[0]);
    if (al)
        tma_load_2d(&S.al[0][0], &M.al, x0 - R - 1, y0 - R, &S.bar[0]);
    tma_load_2d(&S.mk[0][0], &M.mk, x0, y0, &S.bar[0]);
    mbar_expect_tx(&S.bar[1], (unsigned)(sizeof(S.v) + sizeof(S.a) + sizeof(S.im) + (wb ? sizeof(S.wb) : 0) +
                                         (g ? sizeof(S.g) : 0)));
    tma_load_3d(&S.v[0][0], &M.v, 0, x0, y0, &S.bar[1]);
    tma_load_2d(&S.a[0][0], &M.a, x0, y0, &S.bar[1]);
    tma_load_2d(&S.im[0][0], &M.im, x0, y0, &S.bar[1]);
    if (wb)
        tma_load_3d(&S.wb[0][0][0], &M.wb, x0, y0, 0, &S.bar[1]);
    if (g)
        tma_load_3d(&S.g[0][0][0], &M.g, x0, y0, 0, &S.bar[1]);
}

// ------------------------------------------------- pair-symmetric tiles ----
// Newton's third law (f_ji = -f_ij, Eq. 2 and Eq. 34's symmetric weights): a
// CTA whose nodes all hold their 28 bonds evaluates each bond once. Every
// source node i of a bond into the tile (the tile itself, 3 columns to its
// left, 3 rows above, 2 below) evaluates its H+ bonds i -> i + d and stores
// the scalar s of f = s d at the target, s[k][target] for d = d_k; after one
// barrier each tile node adds its own H+ forces (already in registers) and
// gathers -s d of its 14 H- bonds, in the canonical order. Halo sources are
// split into warp-uniform tasks. A CTA in which any bond reached the critical
// stretch (or any node misses a bond) takes the per-warp paths instead.
template <int KR>
struct LatPair {
    alignas(16) float s[lat2d::NP][lat2d::TY * KR][lat2d::TX];
};

// Halo tasks: kind 0 = rows y = p < 0 above the tile (lanes along x), 1 = rows
// y = TYK + p below it, 2 = columns x = p < 0 left of it (lanes along y,
// y = lane - 3); dxs >= 0 restricts a task to the bonds of column dx = dxs.
struct PairTask {
    int kind, p, dxs, warp;
};
__host__ __device__ constexpr bool pair_sel(const PairTask t, const int dx, const int dy)
{
    const bool col = t.dxs < 0 || dx == t.dxs;
    return col && (t.kind == 0 ? dy >= -t.p : t.kind == 1 ? dy <= -1 - t.p : dx >= -t.p);
}
// 36 bonds per lane over 8 warps, at most 5 each (tiles of 16 rows)
constexpr int kPairTasks = 13;
__host__ __device__ constexpr PairTask pair_task(const int i)
{
    constexpr PairTask t[kPairTasks] = {{2, -1, 1, 0}, {2, -1, 2, 1}, {2, -2, 2, 2}, {0, -2, -1, 3},
                                        {0, -3, -1, 3}, {1, 0, -1, 4},  {2, -1, 3, 4}, {0, -1, 0, 5},
                                        {1, 1, -1, 5},  {0, -1, 1, 6},  {0, -1, 2, 6}, {2, -2, 3, 6},
                                        {2, -3, 3, 7}};
    return t[i];
}

template <int KR, bool ALPHA, int TI>
__device__ __forceinline__ void pair_halo_task(const LatStage<KR> &S, LatPair<KR> &P, const Lat2DArgs &A,
                                               const int lane, float2 &wm)
{
    using namespace lat2d;
    constexpr PairTask t = pair_task(TI);
    constexpr int TYK = LatStage<KR>::TYK, HY = LatStage<KR>::HY;
    static_assert(TYK + 5 <= 32, "left-column tasks put the rows on the lanes");
    const int x = t.kind == 2 ? t.p : lane;
    const int y = t.kind == 0 ? t.p : t.kind == 1 ? TYK + t.p : lane - R;
    if (t.kind == 2 && lane >= TYK + 5)
        return;
    const float4 ui = S.u[y + R][x + R];
    const float4 nu = make_float4(-ui.x, -ui.y, -ui.z, -ui.w);
    const float ai = ALPHA ? S.alh()[y + R][x + R] : 0.f;
    static_for<0, NP>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int dx = PDX(k), dy = PDY(k);
        if constexpr (pair_sel(pair_task(TI), dx, dy)) {
            // left-column sources reach rows outside the halo only for targets
            // outside the tile, whose s is never read: clamp the row
            const int hy = t.kind == 2 ? min(max(y + dy + R, 0), HY - 1) : y + dy + R;
            const float4 uj = S.u[hy][x + dx + R];
            const float aj = ALPHA ? S.alh()[hy][x + dx + R] : 0.f;
            float2 fd = make_float2(0.f, 0.f);
            uint32_t md = 0u;
            float2 w = kWatch0;
            const float sb = lattice_bond<dx, dy, ALPHA, false, false>(uj, aj, nu, ai, A, 0u, md, fd, w);
            const bool tgt = x + dx >= 0 && x + dx < TX && y + dy >= 0 && y + dy < TYK;
            if (tgt) {
                P.s[k][y + dy][x + dx] = sb;
                wm.x = fmaxf(wm.x, w.x);
                wm.y = fmaxf(wm.y, w.y);
            }
        }
    });
}

// Pair evaluation of a clean tile: this thread's strip bonds of H+ (forces
// into f, s into P) and its warp's halo tasks; wm collects the break watch.
template <int KR, bool ALPHA>
__device__ __forceinline__ void pair_compute(const LatStage<KR> &S, LatPair<KR> &P, const Lat2DArgs &A,
                                             const float4 (&nu)[KR], const float (&ai)[KR], float2 (&f)[KR],
                                             float2 &wm)
{
    using namespace lat2d;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int hx0 = tx + R, hy0 = ty * KR + R;
    float2 watch[KR];
#pragma unroll
    for (int r = 0; r < KR; ++r)
        watch[r] = kWatch0;
    static_for<0, R + 1>([&](auto dxc) {
        constexpr int dx = decltype(dxc)::value;
        constexpr int ry = RY(dx), lo = PLO(dx);
        asm volatile("" ::: "memory");
        static_for<lo, KR + ry>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const float4 uj = S.u[hy0 + j][hx0 + dx];
            const float aj = ALPHA ? S.alh()[hy0 + j][hx0 + dx] : 0.f;
            static_for<0, KR>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                constexpr int dy = j - r;
                if constexpr (dy >= lo && dy <= ry) {
                    uint32_t md = 0u;
                    const float sb =
                        lattice_bond<dx, dy, ALPHA, false, false>(uj, aj, nu[r], ai[r], A, 0u, md, f[r], watch[r]);
                    const int yt = ty * KR + r + dy;  // the target, if in the tile
                    if (tx + dx < TX && yt >= 0 && yt < KR * TY)
                        P.s[KP(dx, dy)][yt][tx + dx] = sb;
                }
            });
        });
    });
#pragma unroll
    for (int r = 0; r < KR; ++r) {
        wm.x = fmaxf(wm.x, watch[r].x);
        wm.y = fmaxf(wm.y, watch[r].y);
    }
    static_for<0, kPairTasks>([&](auto tc) {
        constexpr int ti = decltype(tc)::value;
        if (pair_task(ti).warp == ty)
            pair_halo_task<KR, ALPHA, ti>(S, P, A, tx, wm);
    });
}

// The 14 H- forces of this thread's strip nodes from their sources' s.
template <int KR>
__device__ __forceinline__ void pair_gather(const LatPair<KR> &P, float2 (&f)[KR])
{
    using namespace lat2d;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    static_for<0, KR>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        static_for<0, NP>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int dx = PDX(k), dy = PDY(k);
            const float s = P.s[k][ty * KR + r][tx];
            lattice_acc<-dx>(f[r].x, s);
            lattice_acc<-dy>(f[r].y, s);
        });
    });
}

// The substep of the tile at (x0, y0) from its staged inputs. On entry this
// thread's group A has landed; group B is awaited with cp.async.wait_group
// WAIT_B before the per-node update. Returns the bonds this thread broke.
// WAIT_B < 0: group B came by tensor copies completing phase parity parB of
// S.bar[1]; if that wait gives up the CTA returns kTileGaveUp at once.
constexpr unsigned kTileGaveUp = ~0u;

// Whether the halo rows of the tile at row y0 carry an Arlequin weight. A
// tile whose halo carries none evaluates every bond with weight 1 exactly, so
// it can skip the weights. Read before the tile's inputs are awaited, so that
// the two loads' latency hides behind the staging.
template <int KR>
__device__ __forceinline__ bool tile_has_alpha(const Lat2DArgs &A, const int y0)
{
    constexpr int HY = LatStage<KR>::HY;
    return A.alpha && A.alpha_rows[min(A.ny, y0 + HY - lat2d::R)] - A.alpha_rows[max(0, y0 - lat2d::R)] > 0;
}

template <bool PMB, int KR, int WAIT_B, bool PAIR = false>
__device__ __forceinline__ unsigned lattice_tile(LatStage<KR> &S, const Lat2DArgs &A, const int x0, const int y0,
                                                 const int init, const bool has_alpha, LatPair<KR> *P = nullptr,
                                                 const unsigned parB = 0)
{
    using namespace lat2d;
    const F32NodeArgs &N = A.nd;
    const int nx = A.nx, ny = A.ny;
    if constexpr (WAIT_B >= 0)
        __syncthreads();  // every thread's asynchronous copies of group A are visible
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int hx0 = tx + R, hy0 = ty * KR + R;
    const int x = x0 + tx, ys = y0 + ty * KR;  // the strip: nodes (x, ys + r), r < KR
    float4 nu[KR];
    float ai[KR];
    float2 watch[KR];
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
        ai[r] = has_alpha ? S.alh()[hy0 + r][hx0] : 0.f;
        f[r] = make_float2(0.f, 0.f);
        watch[r] = kWatch0;
    }
    bool done = false;
    if constexpr (PAIR && !PMB) {
        // every node of the tile in the lattice with all its bonds intact
        const bool clean = __syncthreads_and(full && vbits == (1u << KR) - 1u) != 0;
        if (clean) {
            float2 wm = kWatch0;
            if (has_alpha)
                pair_compute<KR, true>(S, *P, A, nu, ai, f, wm);
            else
                pair_compute<KR, false>(S, *P, A, nu, ai, f, wm);
            // the barrier also publishes every s
            if (__syncthreads_or(N.breaking && watch_bound(wm) >= A.qfast) == 0) {
                pair_gather<KR>(*P, f);
                done = true;
            } else {
#pragma unroll
                for (int r = 0; r < KR; ++r)
                    f[r] = make_float2(0.f, 0.f);
            }
        }
    }
    // Fast path: every node of the warp has all bonds intact; evaluate all
    // bonds without per-bond control flow and only keep the break watch. If a
    // bond may have reached the critical stretch (rare), redo the warp bond by
    // bond.
    bool fast = !done && __all_sync(0xffffffffu, full);
    if (fast) {
        if (has_alpha)
            lattice_strip<KR, true, PMB>(S.u, S.alh(), hy0, hx0, A, nu, ai, m0, m, f, watch);
        else
            lattice_strip<KR, false, PMB>(S.u, S.alh(), hy0, hx0, A, nu, ai, m0, m, f, watch);
        bool hit = false;
#pragma unroll
        for (int r = 0; r < KR; ++r)
            hit = hit || (((vbits >> r) & 1u) && watch_bound(watch[r]) >= A.qfast);
        if (N.breaking && __any_sync(0xffffffffu, hit))
            fast = false;
    }
    if (!fast && !done) {
        if (has_alpha)
            lattice_strip_masked<KR, true, PMB>(S.u, S.alh(), hy0, hx0, A, nu, ai, m0, m, f);
        else
            lattice_strip_masked<KR, false, PMB>(S.u, S.alh(), hy0, hx0, A, nu, ai, m0, m, f);
    }
    if constexpr (WAIT_B >= 0) {
        cp_async_wait<WAIT_B>();  // this thread's group B (its own strip) has landed
    } else {
        const bool ok = mbar_wait(&S.bar[1], parB);  // the tile's group B (tensor copies)
        if (__syncthreads_or(!ok)) {
            tma_gave_up(A);
            mbar_wait(&S.bar[1], parB);
            return kTileGaveUp;
        }
    }
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

// One CTA per tile (grid: tile columns x tile rows); PAIR adds the
// pair-symmetric path (its s table after the stage in shared memory).
template <bool PMB, int KR, int MINB, bool PAIR = false>
__global__ void __launch_bounds__(256, MINB) k_pd_step_lattice2d(const Lat2DArgs A, const int init)
{
    extern __shared__ __align__(16) unsigned char lat_smem[];
    LatStage<KR> &S = *reinterpret_cast<LatStage<KR> *>(lat_smem);
    LatPair<KR> *P = PAIR ? reinterpret_cast<LatPair<KR> *>(lat_smem + sizeof(LatStage<KR>)) : nullptr;
    const int x0 = blockIdx.x * lat2d::TX, y0 = lattice_trow(A, (int)blockIdx.y) * LatStage<KR>::TYK;
    lattice_chain_entry();
    const bool ha = tile_has_alpha<KR>(A, y0);
    lattice_issue_a<KR>(S, A, x0, y0);
    cp_async_commit();
    lattice_issue_b<KR>(S, A, x0, y0);
    cp_async_commit();
    cp_async_wait<1>();
    const unsigned nbroken = lattice_tile<PMB, KR, 0, PAIR>(S, A, x0, y0, init, ha, P);
    count_broken(A.nd.broken, nbroken);
}

// One CTA per tile with the inputs staged by tensor copies. The dynamic
// shared memory is realigned to 128 bytes for the copy destinations.
template <bool PMB, int KR, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pd_step_lattice2d_tma(const Lat2DArgs A,
                                                                      const __grid_constant__ LatMaps M,
                                                                      const int init)
{
    extern __shared__ __align__(16) unsigned char lat_smem[];
    const unsigned off = (128u - (smem_addr(lat_smem) & 127u)) & 127u;
    LatStage<KR> &S = *reinterpret_cast<LatStage<KR> *>(lat_smem + off);
    const int x0 = blockIdx.x * lat2d::TX, y0 = lattice_trow(A, (int)blockIdx.y) * LatStage<KR>::TYK;
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    lattice_chain_entry();
    if (threadIdx.x == 0)
        lattice_tma_issue<KR>(S, M, A, x0, y0);
    const bool ha = tile_has_alpha<KR>(A, y0);
    const bool ok = mbar_wait(&S.bar[0], 0, A.first_polls);
    if (__syncthreads_or(!ok)) {
        tma_gave_up(A);
        mbar_wait(&S.bar[0], 0);
        mbar_wait(&S.bar[1], 0);
        return;
    }
    const unsigned nbroken = lattice_tile<PMB, KR, -1>(S, A, x0, y0, init, ha);
    if (nbroken != kTileGaveUp)
        count_broken(A.nd.broken, nbroken);
}

// Persistent variant with tensor-copy staging: a grid of (SMs x resident
// CTAs) walks the tile list; one thread keeps the next tile of each of the
// two stages in flight while the CTA computes the current one. Stage s is
// used for the CTA's tiles k = s, s + 2, ...: its barriers complete phase
// parity (k / 2) & 1. The same per-tile code, so the same bits.
template <bool PMB, int KR, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pd_step_lattice2d_tpipe(const Lat2DArgs A,
                                                                        const __grid_constant__ LatMaps M,
                                                                        const int init, const int ntiles)
{
    constexpr int TYK = LatStage<KR>::TYK;
    extern __shared__ __align__(16) unsigned char lat_smem[];
    const unsigned off = (128u - (smem_addr(lat_smem) & 127u)) & 127u;
    LatStage<KR> *stages = reinterpret_cast<LatStage<KR> *>(lat_smem + off);
    const int ntx = (A.nx + lat2d::TX - 1) / lat2d::TX;
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&stages[q].bar[0], 1);
            mbar_init(&stages[q].bar[1], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    lattice_chain_entry();
    auto issue = [&](LatStage<KR> &S, const int t) {
        if (t < ntiles)
            lattice_tma_issue<KR>(S, M, A, (t % ntx) * lat2d::TX, lattice_trow(A, t / ntx) * TYK);
    };
    if (threadIdx.x == 0) {
        issue(stages[0], blockIdx.x);
        issue(stages[1], blockIdx.x + G);
    }
    unsigned nbroken = 0;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++k) {
        LatStage<KR> &S = stages[k & 1];
        const unsigned par = (unsigned)(k >> 1) & 1u;
        const int x0 = (t % ntx) * lat2d::TX, y0 = lattice_trow(A, t / ntx) * TYK;
        const bool ha = tile_has_alpha<KR>(A, y0);
        const bool ok = mbar_wait(&S.bar[0], par, A.first_polls);
        if (__syncthreads_or(!ok)) {  // give up: let this tile's and the other stage's copies land first
            tma_gave_up(A);
            mbar_wait(&S.bar[0], par);
            mbar_wait(&S.bar[1], par);
            if (t + G < ntiles) {
                mbar_wait(&stages[(k + 1) & 1].bar[0], (unsigned)((k + 1) >> 1) & 1u);
                mbar_wait(&stages[(k + 1) & 1].bar[1], (unsigned)((k + 1) >> 1) & 1u);
            }
            return;
        }
        const unsigned r = lattice_tile<PMB, KR, -1>(S, A, x0, y0, init, ha, nullptr, par);
        if (r == kTileGaveUp) {
            if (t + G < ntiles) {
                mbar_wait(&stages[(k + 1) & 1].bar[0], (unsigned)((k + 1) >> 1) & 1u);
                mbar_wait(&stages[(k + 1) & 1].bar[1], (unsigned)((k + 1) >> 1) & 1u);
            }
            return;
        }
        nbroken += r;
        __syncthreads();  // every thread is done with S
        if (threadIdx.x == 0)
            issue(S, t + 2 * G);
    }
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
        const int x0 = (t % ntx) * lat2d::TX, y0 = lattice_trow(A, t / ntx) * TYK;
        const bool ha = tile_has_alpha<KR>(A, y0);
        // pending, newest first: B(t+G), A(t+G), B(t); A(t) has landed
        cp_async_wait<3>();
        nbroken += lattice_tile<PMB, KR, 2>(S, A, x0, y0, init, ha);
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
    // raw storage: the argument block is copied in as words (no initialiser runs)
    __shared__ __align__(16) unsigned char sA_raw[sizeof(Lat2DArgs)];
    Lat2DArgs &sA = *reinterpret_cast<Lat2DArgs *>(sA_raw);
    extern __shared__ __align__(16) unsigned char lat_smem[];
    LatStage<KR> &S = *reinterpret_cast<LatStage<KR> *>(lat_smem);
    const int2 w = work[blockIdx.x];
    static_assert(sizeof(Lat2DArgs) % 4 == 0, "argument block copied as words");
    const int *src = reinterpret_cast<const int *>(args + w.x);
    int *dst = reinterpret_cast<int *>(sA_raw);
    for (int q = threadIdx.x; q < (int)(sizeof(Lat2DArgs) / 4); q += blockDim.x)
        dst[q] = src[q];
    __syncthreads();
    const Lat2DArgs &A = sA;
    const int ntx = (A.nx + lat2d::TX - 1) / lat2d::TX;
    const int x0 = (w.y % ntx) * lat2d::TX, y0 = lattice_trow(A, w.y / ntx) * LatStage<KR>::TYK;
    const bool ha = tile_has_alpha<KR>(A, y0);
    lattice_issue_a<KR>(S, A, x0, y0);
    cp_async_commit();
    lattice_issue_b<KR>(S, A, x0, y0);
    cp_async_commit();
    cp_async_wait<1>();
    const unsigned nbroken = lattice_tile<PMB, KR, 0>(S, A, x0, y0, init, ha);
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

template <int KR, int MINB, bool PAIR = false>
cudaError_t launch_lattice_kr(const Lat2DArgs &A0, bool init, cudaStream_t s)
{
    // the pair path serves the linear law; PMB tiles take the per-warp paths
    const size_t smem = sizeof(LatStage<KR>) + (PAIR && !A0.nd.pmb ? sizeof(LatPair<KR>) : 0);
    static int ctas[2] = {0, 0};
    const auto kern =
        A0.nd.pmb ? k_pd_step_lattice2d<true, KR, MINB, false> : k_pd_step_lattice2d<false, KR, MINB, PAIR>;
    cudaError_t e = lattice_prepare(kern, smem, ctas[A0.nd.pmb ? 1 : 0]);
    if (e != cudaSuccess)
        return e;
    Lat2DArgs A = A0;
    const unsigned rows = (unsigned)lattice_tile_rows<LatStage<KR>::TYK>(A, A0);
    const dim3 grid((unsigned)((A.nx + lat2d::TX - 1) / lat2d::TX), rows);
    return lattice_launch(kern, grid, smem, s, A.pdl != 0, A, init ? 1 : 0);
}

// Tensor maps of the inputs of one launch (lattice2d_tma.cu); false when the
// lattice does not meet the copies' alignment (nx % 4 != 0) or encoding failed.
bool lattice_make_maps(const Lat2DArgs &A, int tyk, LatMaps &M);

// Tile configuration with tensor-copy staging; lattices that the copies cannot
// address take the asynchronous-copy kernel of the same shape (same bits).
template <int KR, int MINB>
cudaError_t launch_lattice_tma(const Lat2DArgs &A0, bool init, cudaStream_t s)
{
    LatMaps M;
    if (!lattice_make_maps(A0, LatStage<KR>::TYK, M))
        return launch_lattice_kr<KR, MINB>(A0, init, s);
    constexpr size_t smem = sizeof(LatStage<KR>) + 128;
    static int ctas[2] = {0, 0};
    const auto kern = A0.nd.pmb ? k_pd_step_lattice2d_tma<true, KR, MINB> : k_pd_step_lattice2d_tma<false, KR, MINB>;
    cudaError_t e = lattice_prepare(kern, smem, ctas[A0.nd.pmb ? 1 : 0]);
    if (e != cudaSuccess)
        return e;
    Lat2DArgs A = A0;
    const unsigned rows = (unsigned)lattice_tile_rows<LatStage<KR>::TYK>(A, A0);
    const dim3 grid((unsigned)((A.nx + lat2d::TX - 1) / lat2d::TX), rows);
    return lattice_launch(kern, grid, smem, s, A.pdl != 0, A, M, init ? 1 : 0);
}

// Persistent tensor-copy configuration (falls back like launch_lattice_tma).
template <int KR, int MINB>
cudaError_t launch_lattice_tpipe(const Lat2DArgs &A0, bool init, cudaStream_t s)
{
    LatMaps M;
    if (!lattice_make_maps(A0, LatStage<KR>::TYK, M))
        return launch_lattice_kr<KR, MINB>(A0, init, s);
    constexpr size_t smem = 2 * sizeof(LatStage<KR>) + 128;
    static int ctas[2] = {0, 0};
    const auto kern =
        A0.nd.pmb ? k_pd_step_lattice2d_tpipe<true, KR, MINB> : k_pd_step_lattice2d_tpipe<false, KR, MINB>;
    int &nb = ctas[A0.nd.pmb ? 1 : 0];
    cudaError_t e = lattice_prepare(kern, smem, nb);
    if (e != cudaSuccess)
        return e;
    Lat2DArgs A = A0;
    const int rows = lattice_tile_rows<LatStage<KR>::TYK>(A, A0);
    const int ntiles = ((A.nx + lat2d::TX - 1) / lat2d::TX) * rows;
    const int grid = std::max(1, std::min(ntiles, A.num_sms * nb));
    return lattice_launch(kern, dim3((unsigned)grid), smem, s, A.pdl != 0, A, M, init ? 1 : 0, ntiles);
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
