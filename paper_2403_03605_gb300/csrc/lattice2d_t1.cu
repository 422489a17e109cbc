// lattice2d_t1.cu -- lattice kernel tile configuration 1: strips of 2 nodes per thread (CTA tile 32 x 16
// nodes), at least 4 resident CTAs per SM.
#include "lattice2d.cuh"

namespace pdmts {
cudaError_t launch_lattice2d_t1(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_kr<2, 4>(A, init, s);
}
}  // namespace pdmts
