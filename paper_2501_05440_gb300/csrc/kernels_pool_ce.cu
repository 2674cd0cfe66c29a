// kernels_pool_ce.cu -- the persistent pool kernels instantiated for
// worlds with continuous-energy problems, without time dependence.
#include "pool.cuh"

namespace mcgb {

bool launch_pool_ce(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                   const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st)
{
    return launch_pool_of<false, true>(W, G, Bsrc, Bdst, R, a, pool, grid, st);
}

int pool_occupancy_ce(int pool) { return pool_occupancy_of<true>(pool); }

}  // namespace mcgb
