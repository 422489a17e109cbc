// lattice2d_t0.cu -- lattice kernel tile configuration 0: strips of 2 nodes per thread (CTA tile 32 x 16
// nodes), at least 3 resident CTAs per SM.
#include "lattice2d.cuh"

namespace pdmts {
cudaError_t launch_lattice2d_t0(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_kr<2, 3>(A, init, s);
}
}  // namespace pdmts
