// lattice2d_t3.cu -- lattice kernel tile configuration 3: the persistent pipelined kernel with strips of 1 node per thread
// (CTA tile 32 x 8 nodes), at least 4 resident CTAs per SM.
#include "lattice2d.cuh"

namespace pdmts {
cudaError_t launch_lattice2d_t3(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_pipe<1, 4>(A, init, s);
}
}  // namespace pdmts
