// lattice2d_batch.cu -- the lattice substep batched over several lattices (a
// work list of (instance, tile)), for the tile configurations with one CTA per
// tile (0 and 1).
#include "lattice2d.cuh"

namespace pdmts {
int lattice2d_batch_prepare(Lat2DArgs &A, int tile)
{
    switch (tile) {
    case 0: return lattice_batch_prepare<2, 3>(A);
    case 1: return lattice_batch_prepare<2, 4>(A);
    default: return -1;
    }
}

cudaError_t launch_lattice2d_batch(const Lat2DArgs *d_args, const int2 *d_work, int nwork, int tile, bool pmb,
                                   cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_lattice_batch<2, 3>(d_args, d_work, nwork, pmb, s);
    case 1: return launch_lattice_batch<2, 4>(d_args, d_work, nwork, pmb, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace pdmts
