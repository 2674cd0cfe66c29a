// kernels_pool_mg.cu -- the persistent pool kernels instantiated for
// multigroup worlds without time dependence (the headline lattice).
#include "pool.cuh"

namespace mcgb {

bool launch_pool_mg(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                   const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st)
{
    return launch_pool_of<false, false>(W, G, Bsrc, Bdst, R, a, pool, grid, st);
}

int pool_occupancy_mg(int pool) { return pool_occupancy_of<false>(pool); }

}  // namespace mcgb
