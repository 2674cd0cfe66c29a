// kernels_pool_ce_time.cu -- the persistent pool kernels instantiated for
// worlds with continuous-energy problems and time dependence.
#include "pool.cuh"

namespace mcgb {

bool launch_pool_ce_time(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                   const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st)
{
    return launch_pool_of<true, true>(W, G, Bsrc, Bdst, R, a, pool, grid, st);
}

}  // namespace mcgb
