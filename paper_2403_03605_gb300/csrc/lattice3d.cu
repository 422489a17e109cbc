// lattice3d.cu -- the FP32-bulk PD substep on a regular 3D lattice (arXiv
// 2403.03605, Eq. 1-4 with the Arlequin bond weights of Sec. 3.2 and the
// per-node update of Eq. 38). The family is implicit: a node's neighbours are
// the 122 stencil offsets |d|^2 <= 9 and only its four bond words are read.
//
// One thread per node; a block holds 32 consecutive x of 4 or 8 rows y of one
// plane z, so a warp shares (y, z) and its neighbour loads are coalesced.
// A node's bonds are summed in ascending neighbour-index order, (dz, dy, dx)
// lexicographic, with the sliced-ELL kernel's operations: both give the same
// bits. The stencil is walked row by row ((dz, dy), 29 rows, one rolled loop
// over the set bits of the warp's mask of rows inside the box) into one of
// four compile-time row bodies by the row's reach in dx (0..3), so the code
// stays small. A row's constants and offset come from a 29-row table in
// device memory built once per body (warp-uniform 16-byte loads that stay in
// L1, no indexed constant-bank loads); each row loads through one base
// pointer with the dx offsets as immediates.
//
// Fast path: a warp whose nodes hold every bond that exists evaluates its
// bonds without bit tests. A warp with a lane near the x faces of the box takes a
// variant in which a lane whose x + dx leaves the box reads its own column and
// multiplies that bond's coefficient and stretch by 0 (an exact zero
// contribution). Only the largest reduced stretch (|d + eta|^2 - |d|^2) / |d|^2
// is kept; if it may have reached the critical stretch, or a node of the warp
// misses a bond, the warp evaluates its nodes bond by bond with the bits
// (masked path, the same order and operations, so the same bits when nothing
// breaks).
#include <cstddef>

#include "f32_device.cuh"
#include "lattice2d.cuh"

namespace pdmts {
namespace lat3d {
// offset k of the stencil, in (dz, dy, dx) lexicographic order
struct Off {
    int dx, dy, dz;
};
__host__ __device__ constexpr Off off(const int k)
{
    int c = 0;
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0 || r2 > 9)
                    continue;
                if (c == k)
                    return Off{dx, dy, dz};
                ++c;
            }
    return Off{0, 0, 0};
}
static_assert(off(NS - 1).dz == 3 && off(NS).dz == 0, "122 offsets");
struct OffTable {
    signed char dx[NS], dy[NS], dz[NS];
};
__host__ __device__ constexpr OffTable make_off_table()
{
    OffTable t{};
    for (int k = 0; k < NS; ++k) {
        t.dx[k] = (signed char)off(k).dx;
        t.dy[k] = (signed char)off(k).dy;
        t.dz[k] = (signed char)off(k).dz;
    }
    return t;
}
__constant__ OffTable kOff = make_off_table();
constexpr int stencil_bonds()
{
    int c = 0;
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -reach_y(dz < 0 ? -dz : dz); dy <= reach_y(dz < 0 ? -dz : dz); ++dy)
            c += 2 * reach_x(dz < 0 ? -dz : dz, dy) + 1;
    return c - 1;
}
static_assert(stencil_bonds() == NS, "row bodies cover the stencil");

static_assert(make_row_tab().dz[NR - 1] == 3 && make_row_tab().dz[NR - 2] == 2, "29 rows");
// Rows whose dz (dy) lies in [lo, hi], lo = -3..0, hi = 0..3: entry 4 (lo + 3) + hi.
struct RowMasks {
    uint32_t z[16], y[16];
};
__host__ __device__ constexpr RowMasks make_row_masks()
{
    RowMasks m{};
    const RowTab t = make_row_tab();
    for (int lo = -3; lo <= 0; ++lo)
        for (int hi = 0; hi <= 3; ++hi)
            for (int r = 0; r < NR; ++r) {
                if (t.dz[r] >= lo && t.dz[r] <= hi)
                    m.z[4 * (lo + 3) + hi] |= 1u << r;
                if (t.dy[r] >= lo && t.dy[r] <= hi)
                    m.y[4 * (lo + 3) + hi] |= 1u << r;
            }
    return m;
}
__constant__ RowMasks kRowMasks = make_row_masks();
}  // namespace lat3d

// eta = u_j - u_i from compensated pairs, d . eta (a zero x term of d is left
// out: it changes at most the sign of a zero dot, which no result depends on)
// and lhs = |d + eta|^2 - |d|^2 = 2 d . eta + |eta|^2, for d = (DX, fdy, fdz).
struct Bond3D {
    float e0, e1, e2, dot, lhs;
};
template <int DX>
__device__ __forceinline__ Bond3D bond3d_eval(const float4 s4, const float2 s2, const float4 nu4, const float2 nu2,
                                              const float fdy, const float fdz)
{
    // (dhx, dhy), (dhz, dlx), (dly, dlz): eta = (u_j - u_i)_hi + (u_j - u_i)_lo
    const float2 pa = __fadd2_rn(make_float2(s4.x, s4.y), make_float2(nu4.x, nu4.y));
    const float2 pb = __fadd2_rn(make_float2(s4.z, s4.w), make_float2(nu4.z, nu4.w));
    const float2 pc = __fadd2_rn(s2, nu2);
    Bond3D b;
    b.e0 = __fadd_rn(pa.x, pb.y);
    b.e1 = __fadd_rn(pa.y, pc.x);
    b.e2 = __fadd_rn(pb.x, pc.y);
    float dot;
    if constexpr (DX != 0)
        dot = __fmaf_rn(fdy, b.e1, __fmul_rn((float)DX, b.e0));
    else
        dot = __fmul_rn(fdy, b.e1);
    dot = __fmaf_rn(fdz, b.e2, dot);
    float q = __fmul_rn(b.e0, b.e0);
    q = __fmaf_rn(b.e1, b.e1, q);
    q = __fmaf_rn(b.e2, b.e2, q);
    b.dot = dot;
    b.lhs = __fmaf_rn(2.f, dot, q);
    return b;
}

// Row constants: per |dx| = 0..3 the coefficient c(|xi|) h^2 V, 1/|d|^2,
// |d|^2 and |d| of the bond (dx, dy, dz), for the row's rb = dy^2 + dz^2.
struct Row3D {
    float coef[4], ir2[4], rr[4], rd[4];
};


// Bond (dx, dy, dz) of one node whose row (dy, dz) starts at p4/p2/pa. XE: a
// lane of the warp lies within 3 columns of an x face (xm[dx + 3] = 0 where
// x + dx leaves the box: the lane reads its own column and the bond
// contributes an exact zero).
template <int dx, bool ALPHA, bool PMB, bool XE>
__device__ __forceinline__ void bond3d_node(const float4 *p4, const float2 *p2, const float *pa, const float fdy,
                                            const float fdz, const Row3D &R, const float4 nu4, const float2 nu2,
                                            const float ai, const float (&xm)[7], float (&f)[3], float &qmax)
{
    constexpr int adx = dx < 0 ? -dx : dx;
    const bool in = !XE || xm[dx + 3] != 0.f;
    const float4 s4 = __ldg(in ? p4 + dx : p4);
    const float2 s2 = __ldg(in ? p2 + dx : p2);
    const Bond3D b = bond3d_eval<dx>(s4, s2, nu4, nu2, fdy, fdz);
    float coef = R.coef[adx];
    if constexpr (XE) {
        qmax = fmaxf(qmax, __fmul_rn(__fmul_rn(b.lhs, R.ir2[adx]), xm[dx + 3]));
        coef = __fmul_rn(coef, xm[dx + 3]);
    } else {
        qmax = fmaxf(qmax, __fmul_rn(b.lhs, R.ir2[adx]));
    }
    if constexpr (ALPHA)
        coef = __fmul_rn(coef, bond_weight(ai, __ldg(in ? pa + dx : pa)));
    if constexpr (PMB) {
        const float rr = R.rr[adx];
        const float ry = __fsqrt_rn(__fadd_rn(rr, fmaxf(b.lhs, -rr)));
        const float sc = __fdiv_rn(__fmul_rn(__fmul_rn(coef, rr), b.lhs), __fmul_rn(__fadd_rn(ry, R.rd[adx]), ry));
        f[0] = __fmaf_rn(sc, __fadd_rn((float)dx, b.e0), f[0]);
        f[1] = __fmaf_rn(sc, __fadd_rn(fdy, b.e1), f[1]);
        f[2] = __fmaf_rn(sc, __fadd_rn(fdz, b.e2), f[2]);
    } else {
        const float sc = __fmul_rn(coef, b.dot);
        if constexpr (dx != 0)
            f[0] = __fmaf_rn(sc, (float)dx, f[0]);
        f[1] = __fmaf_rn(sc, fdy, f[1]);
        f[2] = __fmaf_rn(sc, fdz, f[2]);
    }
}

// The bonds of one row (dy, dz) of a node, dx = -RX..RX ascending, loaded
// through one base pointer; RX = 3 is only the centre row (dy = dz = 0),
// which skips dx = 0.
template <int RX, bool ALPHA, bool PMB, bool XE>
__device__ __forceinline__ void row3d(const Lat3DArgs &A, const int row, const float fdy, const float fdz,
                                      const Row3D &R, const float4 nu4, const float2 nu2, const float ai,
                                      const float (&xm)[7], float (&f)[3], float &qmax)
{
    const F32NodeArgs &N = A.nd;
    const float4 *p4 = N.u4_in + row;
    const float2 *p2 = N.u2_in + row;
    const float *pa = ALPHA ? A.alpha + row : nullptr;
    static_for<-RX, RX + 1>([&](auto dxc) {
        constexpr int dx = decltype(dxc)::value;
        if constexpr (!(RX == 3 && dx == 0))
            bond3d_node<dx, ALPHA, PMB, XE>(p4, p2, pa, fdy, fdz, R, nu4, nu2, ai, xm, f, qmax);
    });
}

static_assert(offsetof(Row3DEnt, off) == 64 && offsetof(Row3DEnt, rx) == 76 && sizeof(Row3DEnt) == 80,
              "off, fdy, fdz and rx load as one 16-byte word");
__device__ __forceinline__ void load_row3d(const Row3DEnt &E, Row3D &R, const bool pmb)
{
    const float4 c = __ldg(&E.coef), q = __ldg(&E.ir2);
    R.coef[0] = c.x; R.coef[1] = c.y; R.coef[2] = c.z; R.coef[3] = c.w;
    R.ir2[0] = q.x; R.ir2[1] = q.y; R.ir2[2] = q.z; R.ir2[3] = q.w;
    if (pmb) {
        const float4 rr = __ldg(&E.rr), rd = __ldg(&E.rd);
        R.rr[0] = rr.x; R.rr[1] = rr.y; R.rr[2] = rr.z; R.rr[3] = rr.w;
        R.rd[0] = rd.x; R.rd[1] = rd.y; R.rd[2] = rd.z; R.rd[3] = rd.w;
    }
}

// Fast path of one node: the valid rows of the stencil in ascending (dz, dy)
// (a rolled loop over the set bits of a warp-uniform mask; each row's
// constants come from the row table), each row's bonds in one of four
// compile-time bodies.
template <bool ALPHA, bool PMB, bool XE>
__device__ __forceinline__ void node_fast(const Lat3DArgs &A, const Row3DEnt *rows, const uint32_t valid,
                                          const int i, const int x, const float4 nu4, const float2 nu2,
                                          const float ai, float (&f)[3], float &qmax)
{
    float xm[7];
#pragma unroll
    for (int d = 0; d < 7; ++d)
        xm[d] = (x + d - 3 >= 0 && x + d - 3 < A.nx) ? 1.f : 0.f;
#pragma unroll 1
    for (uint32_t vm = valid; vm != 0u; vm &= vm - 1u) {
        const Row3DEnt &E = rows[__ffs(vm) - 1];
        Row3D R;
        load_row3d(E, R, PMB);
        const int4 m = __ldg(reinterpret_cast<const int4 *>(&E.off));  // off, fdy, fdz, rx
        const int row = i + m.x;
        const float fdy = __int_as_float(m.y), fdz = __int_as_float(m.z);
        switch (m.w) {
        case 3:
            row3d<3, ALPHA, PMB, XE>(A, row, fdy, fdz, R, nu4, nu2, ai, xm, f, qmax);
            break;
        case 2:
            row3d<2, ALPHA, PMB, XE>(A, row, fdy, fdz, R, nu4, nu2, ai, xm, f, qmax);
            break;
        case 1:
            row3d<1, ALPHA, PMB, XE>(A, row, fdy, fdz, R, nu4, nu2, ai, xm, f, qmax);
            break;
        default:
            row3d<0, ALPHA, PMB, XE>(A, row, fdy, fdz, R, nu4, nu2, ai, xm, f, qmax);
            break;
        }
    }
}

// Masked path of one node: its bonds in order with their bits; a bond at or
// past the critical stretch is cleared and carries no force. The operations
// of the fast path, with every term of d . eta present (offsets from a table).
template <bool ALPHA, bool PMB>
__device__ __forceinline__ void node_masked(const Lat3DArgs &A, const int i, const float4 nu4, const float2 nu2,
                                            const float ai, const uint32_t (&m0)[lat3d::W], uint32_t (&m)[lat3d::W],
                                            float (&f)[3])
{
    const F32NodeArgs &N = A.nd;
    const int sy = A.nx, sz = A.nx * A.ny;
#pragma unroll
    for (int w = 0; w < lat3d::W; ++w) {
        const uint32_t word = m0[w];
        uint32_t mw = word;
#pragma unroll 1
        for (int b = 0; b < 32; ++b) {
            const int k = 32 * w + b;
            if (k >= lat3d::NS || !((word >> b) & 1u))
                continue;
            const int dx = lat3d::kOff.dx[k], dy = lat3d::kOff.dy[k], dz = lat3d::kOff.dz[k];
            const int j = i + dx + dy * sy + dz * sz;  // the bond exists: inside the box
            const float4 s4 = __ldg(N.u4_in + j);
            const float2 s2 = __ldg(N.u2_in + j);
            const float fdx = (float)dx, fdy = (float)dy, fdz = (float)dz;
            const float2 pa = __fadd2_rn(make_float2(s4.x, s4.y), make_float2(nu4.x, nu4.y));
            const float2 pb = __fadd2_rn(make_float2(s4.z, s4.w), make_float2(nu4.z, nu4.w));
            const float2 pc = __fadd2_rn(s2, nu2);
            const float e0 = __fadd_rn(pa.x, pb.y), e1 = __fadd_rn(pa.y, pc.x), e2 = __fadd_rn(pb.x, pc.y);
            float dot = __fmul_rn(fdx, e0);
            dot = __fmaf_rn(fdy, e1, dot);
            dot = __fmaf_rn(fdz, e2, dot);
            float q = __fmul_rn(e0, e0);
            q = __fmaf_rn(e1, e1, q);
            q = __fmaf_rn(e2, e2, q);
            const float lhs = __fmaf_rn(2.f, dot, q);
            const int r2 = dx * dx + dy * dy + dz * dz;
            if (N.breaking && lhs >= A.thr[r2]) {
                mw &= ~(1u << b);
                continue;
            }
            float coef = A.coef[r2];
            if constexpr (ALPHA)
                coef = __fmul_rn(coef, bond_weight(ai, __ldg(A.alpha + j)));
            if constexpr (PMB) {
                const float rr = A.r2[r2];
                const float ry = __fsqrt_rn(__fadd_rn(rr, fmaxf(lhs, -rr)));
                const float sc = __fdiv_rn(__fmul_rn(__fmul_rn(coef, rr), lhs), __fmul_rn(__fadd_rn(ry, A.rd[r2]), ry));
                f[0] = __fmaf_rn(sc, __fadd_rn(fdx, e0), f[0]);
                f[1] = __fmaf_rn(sc, __fadd_rn(fdy, e1), f[1]);
                f[2] = __fmaf_rn(sc, __fadd_rn(fdz, e2), f[2]);
            } else {
                const float sc = __fmul_rn(coef, dot);
                f[0] = __fmaf_rn(sc, fdx, f[0]);
                f[1] = __fmaf_rn(sc, fdy, f[1]);
                f[2] = __fmaf_rn(sc, fdz, f[2]);
            }
        }
        m[w] = mw;
    }
}

// Rows of the stencil that stay inside the box for a node in row y of plane
// z: dz in [max(-3, -z), min(3, nz - 1 - z)] and dy likewise.
__device__ __forceinline__ uint32_t valid_rows(const Lat3DArgs &A, const int y, const int z)
{
    return lat3d::kRowMasks.z[4 * (max(-3, -z) + 3) + min(3, A.nz - 1 - z)] &
           lat3d::kRowMasks.y[4 * (max(-3, -y) + 3) + min(3, A.ny - 1 - y)];
}

// Whether every bond of node i that exists is intact (its bond words equal
// the words of its existing bonds).
__device__ __forceinline__ bool all_intact(const Lat3DArgs &A, const int i)
{
    bool full = true;
#pragma unroll
    for (int w = 0; w < lat3d::W; ++w)
        full = full && A.mask[(int64_t)w * A.nd.n + i] == A.exists[(int64_t)w * A.nd.n + i];
    return full;
}

// Masked path of node i with its bond words written back (when `write`);
// returns the number of bonds it broke.
template <bool ALPHA, bool PMB>
__device__ __forceinline__ unsigned node_masked_words(const Lat3DArgs &A, const int i, const float4 nu4,
                                                      const float2 nu2, const float ai, const bool write,
                                                      float (&f)[3])
{
    const int64_t n = A.nd.n;
    uint32_t m0[lat3d::W], m[lat3d::W];
#pragma unroll
    for (int w = 0; w < lat3d::W; ++w)
        m0[w] = A.mask[(int64_t)w * n + i];
    node_masked<ALPHA, PMB>(A, i, nu4, nu2, ai, m0, m, f);
    unsigned nbroken = 0;
    if (write) {
#pragma unroll
        for (int w = 0; w < lat3d::W; ++w)
            if (m[w] != m0[w]) {
                A.mask[(int64_t)w * n + i] = m[w];
                nbroken += __popc(m0[w] ^ m[w]);
            }
    }
    return nbroken;
}

// One thread per node; blocks of 32 x BY nodes (x, y) of one plane z. Blocks
// of 32 x 4 take registers for 9 CTAs per SM (56 per thread: 36 resident
// warps, so a 204,800-node lattice needs 1.22 waves instead of 1.37); blocks
// of 32 x 8 take 64 per thread (32 warps).
template <int BY, bool ALPHA, bool PMB>
__global__ void __launch_bounds__(32 * BY, BY == 4 ? 9 : 4) k_pd_step_lattice3d(const Lat3DArgs A, const int init)
{
    const F32NodeArgs &N = A.nd;
    const int lane = threadIdx.x & 31;
    const int x = blockIdx.x * 32 + lane, y = blockIdx.y * BY + (threadIdx.x >> 5), z = blockIdx.z;
    const Row3DEnt *rows = A.rows;
    lattice_chain_entry();
    if (y >= A.ny)  // the whole warp
        return;
    const int nx = A.nx;
    const bool xin = x < nx;
    // a lane past the box edge mirrors the last column and writes nothing
    const int i = (xin ? x : nx - 1) + nx * (y + A.ny * z);
    const float4 u4 = N.u4_in[i];
    const float2 u2 = N.u2_in[i];
    const float4 nu4 = make_float4(-u4.x, -u4.y, -u4.z, -u4.w);
    const float2 nu2 = make_float2(-u2.x, -u2.y);
    const float ai = ALPHA ? A.alpha[i] : 0.f;
    // a warp whose 7-row neighbourhood carries no weight evaluates every bond
    // with weight 1 exactly and skips the weights
    const bool has_alpha = ALPHA && A.alpha_rows[min(A.ny, y + 4)] - A.alpha_rows[max(0, y - 3)] > 0;
    float f[3] = {0.f, 0.f, 0.f};
    bool fast = __all_sync(0xffffffffu, all_intact(A, i));
    if (fast) {
        float qmax = -INFINITY;
        const bool xe = __any_sync(0xffffffffu, x < 3 || x > nx - 4);
        const uint32_t valid = valid_rows(A, y, z);
        if (has_alpha) {
            if (xe)
                node_fast<true, PMB, true>(A, rows, valid, i, x, nu4, nu2, ai, f, qmax);
            else
                node_fast<true, PMB, false>(A, rows, valid, i, x, nu4, nu2, ai, f, qmax);
        } else {
            if (xe)
                node_fast<false, PMB, true>(A, rows, valid, i, x, nu4, nu2, ai, f, qmax);
            else
                node_fast<false, PMB, false>(A, rows, valid, i, x, nu4, nu2, ai, f, qmax);
        }
        if (N.breaking && __any_sync(0xffffffffu, xin && qmax >= A.qfast))
            fast = false;
    }
    unsigned nbroken = 0;
    if (!fast) {
        f[0] = f[1] = f[2] = 0.f;
        nbroken = has_alpha ? node_masked_words<true, PMB>(A, i, nu4, nu2, ai, xin, f)
                            : node_masked_words<false, PMB>(A, i, nu4, nu2, ai, xin, f);
    }
    count_broken(N.broken, nbroken);
    if (!xin)
        return;
    float uh[3] = {u4.x, u4.y, u4.z}, ul[3] = {u4.w, u2.x, u2.y};
    finish_node_f32<3>(N, i, f, uh, ul, init);
}

template <int BY>
static cudaError_t launch_lattice3d_by(const Lat3DArgs &A, bool init, cudaStream_t s)
{
    const dim3 grid((unsigned)((A.nx + 31) / 32), (unsigned)((A.ny + BY - 1) / BY), (unsigned)A.nz);
    const bool al = A.alpha != nullptr;
    const auto kern = al ? (A.nd.pmb ? k_pd_step_lattice3d<BY, true, true> : k_pd_step_lattice3d<BY, true, false>)
                         : (A.nd.pmb ? k_pd_step_lattice3d<BY, false, true> : k_pd_step_lattice3d<BY, false, false>);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(32 * BY);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = A.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, A, init ? 1 : 0);
}

cudaError_t launch_pd_step_lattice3d(const Lat3DArgs &A, bool init, cudaStream_t s)
{
    if (A.nx <= 0 || A.ny <= 0 || A.nz <= 0)
        return cudaSuccess;
    if ((A.ny + 3) / 4 > 65535 || A.nz > 65535)
        return cudaErrorInvalidConfiguration;
    return A.tile == 1 ? launch_lattice3d_by<8>(A, init, s) : launch_lattice3d_by<4>(A, init, s);
}

}  // namespace pdmts
