// lattice3d.cu -- the FP32-bulk PD substep on a regular 3D lattice (arXiv
// 2403.03605, Eq. 1-4 with the Arlequin bond weights of Sec. 3.2 and the
// per-node update of Eq. 38). The family is implicit: a node's neighbours are
// the 122 stencil offsets, visited in ascending neighbour-index order, and
// only its four bond words are read. One thread per node; the neighbours'
// displacements come through the read-only cache. Every operation and its
// order follow the sliced-ELL FP32 kernel, so the two give the same bits.
#include "f32_device.cuh"
#include "lattice2d.cuh"

namespace pdmts {
namespace lat3d {
struct Off {
    int dx, dy, dz;
};
// offset k of the stencil: (dz, dy, dx) lexicographic, 0 < |d|^2 <= 9
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
}  // namespace lat3d

// f += s d for a compile-time component d (skipped when 0: f + 0 s == f)
template <int D>
__device__ __forceinline__ void acc3(float &f, const float s)
{
    if constexpr (D != 0)
        f = __fmaf_rn(s, (float)D, f);
}

template <bool ALPHA, bool PMB>
__global__ void __launch_bounds__(256) k_pd_step_lattice3d(const Lat3DArgs A, const int init)
{
    const F32NodeArgs &N = A.nd;
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5), z = blockIdx.z;
    const bool valid = x < A.nx && y < A.ny;
    const int sy = A.nx, sz = A.nx * A.ny;  // n < 2^24 on this path
    const int i = valid ? x + sy * y + sz * z : 0;
    lattice_chain_entry();
    const float4 u4 = N.u4_in[i];
    const float2 u2 = N.u2_in[i];
    const float4 nu4 = make_float4(-u4.x, -u4.y, -u4.z, -u4.w);
    const float2 nu2 = make_float2(-u2.x, -u2.y);
    const float ai = ALPHA ? A.alpha[i] : 0.f;
    uint32_t m0[lat3d::W], m[lat3d::W];
#pragma unroll
    for (int w = 0; w < lat3d::W; ++w) {
        m0[w] = valid ? A.mask[(int64_t)w * N.n + i] : 0u;
        m[w] = m0[w];
    }
    float f[3] = {0.f, 0.f, 0.f};
    static_for<0, lat3d::NS>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr lat3d::Off o = lat3d::off(k);
        constexpr int w = k >> 5, b = k & 31, r2 = o.dx * o.dx + o.dy * o.dy + o.dz * o.dz;
        if ((m0[w] >> b) & 1u) {
            const int j = i + o.dx + o.dy * sy + o.dz * sz;
            const float4 j4 = __ldg(N.u4_in + j);
            const float2 j2 = __ldg(N.u2_in + j);
            // (dhx, dhy), (dhz, dlx), (dly, dlz): eta = (u_j - u_i)_hi + (u_j - u_i)_lo
            const float2 pa = __fadd2_rn(make_float2(j4.x, j4.y), make_float2(nu4.x, nu4.y));
            const float2 pb = __fadd2_rn(make_float2(j4.z, j4.w), make_float2(nu4.z, nu4.w));
            const float2 pc = __fadd2_rn(j2, nu2);
            const float eta[3] = {__fadd_rn(pa.x, pb.y), __fadd_rn(pa.y, pc.x), __fadd_rn(pb.x, pc.y)};
            // d . eta and |eta|^2 in the sliced-ELL kernel's order
            float dot = __fmul_rn((float)o.dx, eta[0]);
            dot = __fmaf_rn((float)o.dy, eta[1], dot);
            dot = __fmaf_rn((float)o.dz, eta[2], dot);
            float e2 = __fmul_rn(eta[0], eta[0]);
            e2 = __fmaf_rn(eta[1], eta[1], e2);
            e2 = __fmaf_rn(eta[2], eta[2], e2);
            const float lhs = __fmaf_rn(2.f, dot, e2);
            if (N.breaking && lhs >= A.thr[r2]) {
                m[w] &= ~(1u << b);
            } else {
                float coef = A.coef[r2];
                if constexpr (ALPHA)
                    coef = __fmul_rn(coef, bond_weight(ai, __ldg(A.alpha + j)));
                if constexpr (PMB) {
                    const float rr = A.r2[r2];
                    const float ry = __fsqrt_rn(__fadd_rn(rr, fmaxf(lhs, -rr)));
                    const float sc = __fdiv_rn(__fmul_rn(__fmul_rn(coef, rr), lhs), __fmul_rn(__fadd_rn(ry, A.rd[r2]), ry));
                    f[0] = __fmaf_rn(sc, __fadd_rn((float)o.dx, eta[0]), f[0]);
                    f[1] = __fmaf_rn(sc, __fadd_rn((float)o.dy, eta[1]), f[1]);
                    f[2] = __fmaf_rn(sc, __fadd_rn((float)o.dz, eta[2]), f[2]);
                } else {
                    const float sc = __fmul_rn(coef, dot);
                    acc3<o.dx>(f[0], sc);
                    acc3<o.dy>(f[1], sc);
                    acc3<o.dz>(f[2], sc);
                }
            }
        }
    });
    unsigned nbroken = 0;
#pragma unroll
    for (int w = 0; w < lat3d::W; ++w)
        if (m[w] != m0[w]) {
            A.mask[(int64_t)w * N.n + i] = m[w];
            nbroken += __popc(m0[w] ^ m[w]);
        }
    count_broken(N.broken, nbroken);
    if (!valid)
        return;
    float uh[3] = {u4.x, u4.y, u4.z}, ul[3] = {u4.w, u2.x, u2.y};
    finish_node_f32<3>(N, i, f, uh, ul, init);
}

cudaError_t launch_pd_step_lattice3d(const Lat3DArgs &A, bool init, cudaStream_t s)
{
    if (A.nx <= 0 || A.ny <= 0 || A.nz <= 0)
        return cudaSuccess;
    if (A.nz > 65535 || (A.ny + 7) / 8 > 65535)
        return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)((A.nx + 31) / 32), (unsigned)((A.ny + 7) / 8), (unsigned)A.nz);
    const bool al = A.alpha != nullptr;
    const auto kern = al ? (A.nd.pmb ? k_pd_step_lattice3d<true, true> : k_pd_step_lattice3d<true, false>)
                         : (A.nd.pmb ? k_pd_step_lattice3d<false, true> : k_pd_step_lattice3d<false, false>);
    return lattice_launch(kern, grid, 0, s, A.pdl != 0, A, init ? 1 : 0);
}

}  // namespace pdmts
