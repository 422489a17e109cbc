// lattice2d_tma.cu -- tensor maps of the lattice kernel's inputs for the
// tensor-copy staging (tile configurations 5 to 8), and their launchers.
#include <cudaTypedefs.h>

#include "lattice2d.cuh"

namespace pdmts {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// One map: `rank` dims (innermost first), byte strides of dims 1.., box.
static bool encode(CUtensorMap &m, CUtensorMapDataType type, const void *base, const int rank,
                   const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box)
{
    const cuuint32_t es[3] = {1, 1, 1};
    return encode_fn()(&m, type, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool lattice_make_maps(const Lat2DArgs &A, const int tyk, LatMaps &M)
{
    using namespace lat2d;
    const cuuint64_t nx = (cuuint64_t)A.nx, ny = (cuuint64_t)A.ny, n = (cuuint64_t)A.nd.n;
    if (A.nx % 4 != 0 || !encode_fn() || n != nx * ny)
        return false;
    const cuuint32_t hy = (cuuint32_t)(tyk + 2 * R);
    bool ok = true;
    {  // u: float4 per node as 4 FP32 components, halo box
        const cuuint64_t d[3] = {4, nx, ny}, st[2] = {16, 16 * nx};
        const cuuint32_t b[3] = {4, (cuuint32_t)HX, hy};
        ok = ok && encode(M.u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A.nd.u4_in, 3, d, st, b);
    }
    {  // v: float4 per node, tile box
        const cuuint64_t d[3] = {4, nx, ny}, st[2] = {16, 16 * nx};
        const cuuint32_t b[3] = {4, (cuuint32_t)TX, (cuuint32_t)tyk};
        ok = ok && encode(M.v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A.nd.v4, 3, d, st, b);
    }
    {  // a: float2 per node copied as one 8-byte word
        const cuuint64_t d[2] = {nx, ny}, st[1] = {8 * nx};
        const cuuint32_t b[2] = {(cuuint32_t)TX, (cuuint32_t)tyk};
        ok = ok && encode(M.a, CU_TENSOR_MAP_DATA_TYPE_UINT64, A.nd.a, 2, d, st, b);
    }
    const cuuint64_t d2[2] = {nx, ny}, st2[1] = {4 * nx};
    const cuuint32_t bt[2] = {(cuuint32_t)TX, (cuuint32_t)tyk};
    ok = ok && encode(M.mk, CU_TENSOR_MAP_DATA_TYPE_UINT32, A.mask, 2, d2, st2, bt);
    ok = ok && encode(M.im, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A.nd.inv_m, 2, d2, st2, bt);
    M.al = M.u;
    if (A.alpha) {  // weight halo from column x0 - R - 1, HX + 2 wide
        const cuuint32_t b[2] = {(cuuint32_t)HXA, hy};
        ok = ok && encode(M.al, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A.alpha, 2, d2, st2, b);
    }
    const cuuint64_t d3[3] = {nx, ny, 2}, st3[2] = {4 * nx, 4 * n};
    const cuuint32_t b3[3] = {(cuuint32_t)TX, (cuuint32_t)tyk, 2};
    M.wb = M.u;
    M.g = M.u;
    if (A.nd.wb)
        ok = ok && encode(M.wb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A.nd.wb, 3, d3, st3, b3);
    if (A.nd.g)
        ok = ok && encode(M.g, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A.nd.g, 3, d3, st3, b3);
    return ok;
}

cudaError_t launch_lattice2d_t5(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_tma<2, 4>(A, init, s);
}

cudaError_t launch_lattice2d_t6(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_tma<2, 3>(A, init, s);
}

cudaError_t launch_lattice2d_t7(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_tpipe<2, 2>(A, init, s);
}

cudaError_t launch_lattice2d_t8(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_tpipe<1, 4>(A, init, s);
}

cudaError_t launch_lattice2d_t9(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_tma<4, 2>(A, init, s);
}

}  // namespace pdmts
