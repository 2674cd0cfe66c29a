// kernels_pool.cu -- dispatch to the persistent pool kernels (pool.cuh): the
// instantiation without continuous-energy physics when the world has none, and
// the one without the particle clock when nothing is time dependent.
#include "kernels.h"

namespace mcgb {

bool launch_pool_mg(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                    const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st);
bool launch_pool_mg_time(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                         const RunBufs &R, const PersistentArgs &a, int pool, int grid,
                         cudaStream_t st);
bool launch_pool_ce(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                    const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st);
bool launch_pool_ce_time(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                         const RunBufs &R, const PersistentArgs &a, int pool, int grid,
                         cudaStream_t st);
int pool_occupancy_mg(int pool);
int pool_occupancy_ce(int pool);

int pool_threads() { return 256; }

int pool_particles_per_block(int pool)
{
    return pool < 256 ? pool * 4 : (pool > 2000 ? pool - 2000 : pool);
}

int pool_max_blocks_per_sm(int pool, bool ce)
{
    return ce ? pool_occupancy_ce(pool) : pool_occupancy_mg(pool);
}

bool launch_pool(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                 const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st)
{
    if (W.ce_any)
        return W.time_any ? launch_pool_ce_time(W, G, Bsrc, Bdst, R, a, pool, grid, st)
                          : launch_pool_ce(W, G, Bsrc, Bdst, R, a, pool, grid, st);
    return W.time_any ? launch_pool_mg_time(W, G, Bsrc, Bdst, R, a, pool, grid, st)
                      : launch_pool_mg(W, G, Bsrc, Bdst, R, a, pool, grid, st);
}

}  // namespace mcgb
