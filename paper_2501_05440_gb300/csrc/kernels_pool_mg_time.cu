// kernels_pool_mg_time.cu -- the persistent pool kernels instantiated for
// multigroup worlds with time dependence.
#include "pool.cuh"

namespace mcgb {

bool launch_pool_mg_time(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                   const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st)
{
    return launch_pool_of<true, false>(W, G, Bsrc, Bdst, R, a, pool, grid, st);
}

}  // namespace mcgb
