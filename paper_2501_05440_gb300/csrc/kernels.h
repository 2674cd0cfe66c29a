// kernels.h -- host-side launchers of the library's kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "world.h"

namespace mcgb {

// ---- event mode (one kernel per event type) -------------------------------
// Births of every slot of a generation into P (gen_dev: the cycle index is read
// there when not null, for graph replay).  The event forms start from these;
// the persistent kernels take their births from them too (PersistentArgs::preborn).
void launch_source(const World &W, const Particles &P, const Bank &Bsrc, const RunBufs &R, int gen,
                   int64_t total, const int64_t *gen_base, const int *src_idx, int eigen, int block,
                   cudaStream_t st, const int *gen_dev = nullptr);
// Algorithmic state bytes one particle moves in a k_advance launch over the
// identity list: the fields loaded and stored, the flight's event queue entry.
double event_advance_bytes(const World &W);
void launch_advance(const World &W, const Particles &P, const RunBufs &R, const int *list, int n,
                    const int *n_dev, int *q_cross, int *q_coll, int block, cudaStream_t st);
void launch_cross(const World &W, const Particles &P, const RunBufs &R, const int *q_cross,
                  int n_bound, int *next, int *next_n, int block, cudaStream_t st);
void launch_collide(const World &W, const Particles &P, const Bank &Bdst, const RunBufs &R,
                    const int *q_coll, int n_bound, int *next, int *next_n, int block,
                    cudaStream_t st);
void launch_segment(const World &W, const Particles &P, const Bank &Bdst, const RunBufs &R,
                    const int *list, int n, const int *n_dev, int *next, int *next_n, int block,
                    cudaStream_t st);

// ---- persistent event loop -------------------------------------------------
struct PersistentArgs {
    int64_t total;           // work items (slots) when gen_n is null
    const int *gen_n;        // device total (bank size) when not null
    int *work;               // device work counter (zeroed before the launch)
    long long max_passes;    // > 0: a block (warp) stops after this many passes of its event
                             // loop and raises ERR_ITER (histories left unfinished)
};
// The persistent kernels take each slot's birth from the particle arrays, where
// launch_source made it for the whole generation before their launch.
// births read Bsrc (the previous cycle's bank), new sites are appended to Bdst
void launch_persistent(const World &W, const Particles &P, const Bank &Bsrc, const Bank &Bdst,
                       const RunBufs &R, const PersistentArgs &a, int grid, int block,
                       cudaStream_t st);
int persistent_max_blocks_per_sm(int block);
// sorted-pool variants in shared memory: `pool` = 256, 512 or 1024 particles per
// block sorted block-wide, or 32, 64 or 128 particles per warp sorted per warp
bool launch_pool(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                 const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st);
// resident blocks per SM of a pool variant (ce: the instantiation with
// continuous-energy physics, which runs with fewer blocks)
int pool_max_blocks_per_sm(int pool, bool ce);
int pool_threads();
int pool_particles_per_block(int pool);

// ---- end of cycle / generation --------------------------------------------
// Exclusive scan of n counts into out; *total = sum.  scratch holds one int per
// 4096 inputs (scan_scratch_ints(n)).
int64_t scan_scratch_ints(int64_t n);
void scan_exclusive(const int *in, int *out, int64_t n, int *total, int *scratch, cudaStream_t st);
void launch_perm(const Bank &B, const int *off, const int *M, int *perm, int grid, cudaStream_t st);
void launch_resample(const int *perm, const int *M, int64_t N, double xi, int *src_idx,
                     int *err, int64_t cap, cudaStream_t st);
// sums over slots [0, total): k estimators into kout[2] (kout[2 * *cyc_dev ..] when
// cyc_dev is given), counters into cnt[5]
void launch_reduce_gen(const Particles &P, int64_t total, const int *total_dev, double *kout,
                       unsigned long long *cnt, cudaStream_t st, const int *cyc_dev = nullptr);
void launch_tally_cycle(double *tacc, int acc_size, int nrep, double n, int active,
                        double *tsum, double *tsum2, cudaStream_t st, const int *cyc_dev = nullptr,
                        int inactive = 0);
// resampling with the draw of the cycle read on the device: xi_tab[*cyc_dev]
void launch_resample_dev(const int *perm, const int *M, int64_t N, const double *xi_tab,
                         const int *cyc_dev, int *src_idx, int *err, int64_t cap, cudaStream_t st);
// end of a replayed cycle: bank size into bank_m[*cyc], then ++*cyc
void launch_cycle_end(int *cyc_dev, const int *M, int64_t *bank_m, cudaStream_t st);
void launch_acc_reduce(const double *tacc, int acc_size, int nrep, double *out, cudaStream_t st);
// sharded power iteration: pack the rank's ordered sites, resample its next
// sources from the global bank, fold the all-rank sums into the statistics
void launch_pack_sites(const Bank &B, const int *perm, int64_t M, int64_t j0, ShardSite *out,
                       cudaStream_t st);
void launch_unpack_sources(const ShardSite *bank, int64_t M, int64_t N, int64_t j0, int64_t n,
                           double xi, const Bank &Bs, cudaStream_t st);
void launch_sites_to_bank(const ShardSite *in, int64_t n, const Bank &Bs, cudaStream_t st);
void launch_shard_stats(const double *sums, int acc_size, double N, int cyc, int active,
                        double *kout, double *tsum, double *tsum2, cudaStream_t st);
// spatial domain decomposition (kernels_domain.cu)
void launch_dom_sources(const World &W, const Particles &P, int gen, int64_t N,
                        const ShardSite *bank, int64_t M, double xi, const DomainCut &dom,
                        const double *cuts, int nd, int rank, int *list, int *n_list, int *err,
                        cudaStream_t st);
void launch_dom_sweep(const World &W, const Particles &P, const Bank &Bdst, const RunBufs &R,
                      const int *list, int n, int *work, const DomainCut &dom, int *outbox,
                      int *n_out, int grid, cudaStream_t st);
void launch_dom_pack(const Particles &P, const int *outbox, int n, const DomainCut &dom, int rank,
                     FlightRec *out, cudaStream_t st);
void launch_dom_unpack(const World &W, const Particles &P, const FlightRec *in, int64_t n, int rank,
                       int *list, int *n_list, cudaStream_t st);
void launch_dom_reduce(const Particles &P, int64_t N, double *ksum, unsigned long long *cnt,
                       int *nfis_out, cudaStream_t st);
void launch_dom_sites(const Bank &B, int64_t m, ShardSite *out, cudaStream_t st);
void launch_dom_place(const ShardSite *in, int64_t m, const int *off, ShardSite *glob, int64_t cap,
                      int *err, cudaStream_t st);
void launch_dom_records(const Particles &P, int64_t N, int *nc, int *nx, int *nf, int *fate, int *g,
                        unsigned long long *rng, cudaStream_t st);
void launch_gen_base(const int64_t *base, int nprob, const int *off, const int *M,
                     int64_t *next_base, cudaStream_t st);
void launch_copy_records(const Particles &P, int64_t n, int *ncoll, int *ncross, uint64_t *rng,
                         int *nfis, int *fate, int *g, cudaStream_t st);

// ---- building blocks for checks ---------------------------------------------
void launch_rng_states(uint64_t seed, uint64_t first_id, int64_t n, int draws, uint64_t *out,
                       cudaStream_t st);
void launch_log(const World &W, int64_t n, const double *xi, double *out, cudaStream_t st);
void launch_fpint_ops(int64_t n, const double *a, const double *b, double *out, cudaStream_t st);
// FP64 throughput probe: grid blocks of 256 threads, fp64_rate_chains() FMAs per
// thread per iteration
void launch_fp64_rate(int grid, long long iters, double *sink, cudaStream_t st);
int fp64_rate_chains();
void launch_probe(const World &W, int root_univ, int64_t n, const double *pos, const double *dir,
                  int *path, double *dist, int *kind, cudaStream_t st);
void launch_ce_lookup(const World &W, int mat, int64_t n, const double *E, double *out,
                      cudaStream_t st);

// ---- derivatives (likelihood-ratio replay) --------------------------------
struct ReplayArgs {
    int gen;
    int64_t n;               // slots of this generation
    const int *site;         // bank site per slot for gen > 0 (sorted bank copy index), or null
    const Bank *bank;        // start states of this generation (gen > 0)
    const double *own;       // per-slot detector tally by group, this generation
    const double *w;         // weights [G]
    const double *sub_next;  // subtree totals of the next generation's slots (or null)
    const int *off;          // first child slot of each slot in the next generation
    const int *nfis;         // children per slot
    int det_cell;
    int G, nmat;
    double *grad;            // [nmat*G*(G+2)] accumulators
};
void launch_subtree(const double *own, const double *w, int G, int64_t n, const double *sub_next,
                    const int *off, const int *nfis, double *sub, cudaStream_t st);
void launch_replay(const World &W, const ReplayArgs &a, int block, cudaStream_t st);
// device-pointer derivative path: new multigroup tables written in place
// (*bad set on invalid input), detector tally sums, scaling
void launch_update_mg(const World &W, int first, int nmat, int G, const double *sigt,
                      const double *sigs, const double *nusf, int *bad, cudaStream_t st);
void launch_own_sum(const double *own, int64_t n, int G, int accumulate, double *out,
                    cudaStream_t st);
void launch_scale(const double *src, int64_t n, double N, double *dst, cudaStream_t st);

}  // namespace mcgb
