// lattice2d_t4.cu -- lattice kernel tile configuration 4: strips of 2 nodes per thread (CTA tile 32 x 16
// nodes), 3 resident CTAs per SM, each bond of a clean tile evaluated once (pair-symmetric path).
#include "lattice2d.cuh"

namespace pdmts {
cudaError_t launch_lattice2d_t4(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_kr<2, 3, true>(A, init, s);
}
}  // namespace pdmts
