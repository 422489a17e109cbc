// lattice2d_t2.cu -- lattice kernel tile configuration 2: the persistent pipelined kernel with strips of 2 nodes per thread
// (CTA tile 32 x 16 nodes), at least 2 resident CTAs per SM.
#include "lattice2d.cuh"

namespace pdmts {
cudaError_t launch_lattice2d_t2(const Lat2DArgs &A, bool init, cudaStream_t s)
{
    return launch_lattice_pipe<2, 2>(A, init, s);
}
}  // namespace pdmts
