/*
 * mcgb.h -- C ABI of the GB300 event-based Monte Carlo neutral-particle
 * transport library (libmcgb.so).
 *
 * The calls follow the paper's statement of the problem (arXiv 2501.05440,
 * Sec. 1): materials with multigroup or pointwise (continuous-energy) cross
 * sections, constructive-solid-geometry cells bounded by surfaces and tracked
 * surface to surface, a source, N particles run for C k-eigenvalue cycles or
 * as a fixed-source problem, and track-length tallies and k read back.  Sec. 2
 * describes the event-based GPU scheme these calls drive: particles repeatedly
 * sample a distance to collision, find the nearest surface, move, score and
 * then cross or collide.
 *
 * Conventions
 *  - Every call returns int: MCGB_OK (0) or a negative MCGB_E_* code; a message
 *    for the last failure on the calling thread is in mcgb_last_error().
 *  - Input arrays are host pointers and are copied; the caller keeps
 *    ownership.  Output arrays are caller-allocated host buffers with a
 *    capacity; when it is too small the call returns MCGB_E_INVALID_ARG and
 *    writes the required element count to *needed (when needed is not NULL).
 *  - Everything runs on the context's CUDA device and stream.  Problem tables
 *    are uploaded at the first run after a change; all transport steps run in
 *    this library's kernels (there is no CPU fallback; without a usable CUDA
 *    device mcgb_create fails with MCGB_E_CUDA).
 *  - Floating point is IEEE double throughout (the paper uses double
 *    precision for all floating-point operations, Sec. 5).
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef MCGB_H
#define MCGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcgb_ctx mcgb_ctx;
typedef struct mcgb_batch mcgb_batch;

/* status codes */
enum {
    MCGB_OK = 0,
    MCGB_E_INVALID_ARG = -1,   /* bad argument, or output capacity too small */
    MCGB_E_STATE = -2,         /* call out of order (e.g. no source), empty bank */
    MCGB_E_CUDA = -3,          /* CUDA runtime error or no device */
    MCGB_E_OOM = -4,           /* device allocation failed */
    MCGB_E_BANK_OVERFLOW = -5, /* more fission sites than the bank holds */
    MCGB_E_LOST_PARTICLES = -6,/* more than 1e-6 of histories found no cell */
    MCGB_E_TIMEOUT = -7,       /* iteration or generation limit reached */
    MCGB_E_NOT_FOUND = -8      /* unknown id */
};

/* geometry vocabulary */
enum { MCGB_SURF_PX = 0, MCGB_SURF_PY = 1, MCGB_SURF_PZ = 2, MCGB_SURF_PLANE = 3,
       MCGB_SURF_CYLZ = 4, MCGB_SURF_SPHERE = 5 };
enum { MCGB_BC_NONE = 0, MCGB_BC_VACUUM = 1, MCGB_BC_REFLECT = 2 };
enum { MCGB_FILL_MATERIAL = 0, MCGB_FILL_LATTICE = 1 };
/* sources */
enum { MCGB_SRC_BOX = 0, MCGB_SRC_POINT = 1 };
enum { MCGB_ACCEPT_ANY = 0, MCGB_ACCEPT_FISSILE = 1 };
enum { MCGB_ENERGY_CHI = 0, MCGB_ENERGY_PDF = 1, MCGB_ENERGY_FIXED = 2, MCGB_ENERGY_MAXWELL = 3 };
enum { MCGB_DIR_ISO = 0, MCGB_DIR_BEAM = 1 };
/* tally filters */
enum { MCGB_FILTER_CELL = 0, MCGB_FILTER_LATTICE = 1, MCGB_FILTER_MATERIAL = 2 };
/* execution modes */
enum { MCGB_MODE_EVENT = 0,       /* one kernel per event type, host-driven loop */
       MCGB_MODE_PERSISTENT = 1,  /* one grid-resident event loop per cycle, CUDA graph */
       MCGB_MODE_SEGMENT = 2 };   /* the monolithic event design of Sec. 2: one kernel per
                                     segment (flight, then the crossing or collision it
                                     ends in) for every live particle, unsorted, with two
                                     alternating particle lists; host-driven loop */

/* Options.  Zero-initialised fields take defaults. */
typedef struct {
    int device;             /* CUDA device ordinal (default 0) */
    int mode;               /* MCGB_MODE_* (default MCGB_MODE_EVENT) */
    int block;              /* threads per block (default: autotuned or 128) */
    int blocks_per_sm;      /* persistent mode: resident blocks per SM (default: occupancy) */
    int record_histories;   /* keep per-history records of the last cycle / generation 0 */
    double bank_factor;     /* fission bank capacity as a multiple of N (default 3) */
    int max_iterations;     /* event / segment mode: host loop iterations per cycle or
                               generation (default 1e7); persistent mode: passes of each
                               block's (or warp's) event loop per launch (default none).
                               Reaching it fails the run with MCGB_E_TIMEOUT, the
                               unfinished histories abandoned; the context stays usable */
    int pool;               /* persistent mode: particles held in shared memory and run
                               event type by event type from sorted lists: 256 (one per
                               thread, four resident blocks per SM), 512 or 1024 per
                               256-thread block; 2256 or 2512 for 256 or 512 per
                               128-thread block; 32, 64 or 128 per warp (warp-level
                               lists, no block barriers); 0 = default (2256 for
                               multigroup worlds, 256 for continuous energy, 512 for
                               continuous energy with time dependence); -1 = one
                               particle per thread in registers */
    int graphs;             /* persistent mode: run every eigenvalue cycle after the first
                               as one CUDA graph launch, with no host synchronisation
                               between cycles (0 = on, -1 = off) */
} mcgb_opts;

/* Event and history counters of the last run. */
typedef struct {
    int64_t histories, collisions, crossings, leaks, lost, capped, generations;
    int64_t kernel_launches;   /* kernels this library launched during the run */
    int64_t event_iterations;  /* event / segment mode: host loop iterations */
    int64_t world_bytes;       /* bytes of problem tables uploaded to the device */
    int64_t time_cut;          /* histories that reached the time cutoff */
} mcgb_counters;

/* Launch shape chosen by the autotuner for a batch. */
typedef struct {
    int block;              /* threads per block (register-resident variant) */
    int blocks_per_sm;      /* resident blocks per SM in the persistent launch */
    int pool;               /* particles per block in shared memory, -1 = register variant */
    double ms;              /* measured time of the tuning run */
} mcgb_tune;

/* --------------------------------------------------------------------------- */
/* context                                                                      */
/* Create a context on opts->device (opts may be NULL).  Fails with MCGB_E_CUDA
 * when no CUDA device is usable. */
int mcgb_create(mcgb_ctx **out, const mcgb_opts *opts);
int mcgb_destroy(mcgb_ctx *ctx);
/* Message for the last failing call on this thread (never NULL). */
const char *mcgb_last_error(void);
/* Run subsequent work on this cudaStream_t (NULL = the legacy default stream). */
int mcgb_set_stream(mcgb_ctx *ctx, void *cuda_stream);
int mcgb_set_mode(mcgb_ctx *ctx, int mode);

/* --------------------------------------------------------------------------- */
/* geometry: constructive solid geometry with surface tracking (Sec. 1)          */
/* Surface f(r) = 0 with coef: PX/PY/PZ {x0}; PLANE {a,b,c,d} (a x + b y + c z = d);
 * CYLZ {x0, y0, R}; SPHERE {x0, y0, z0, R}.  bc: MCGB_BC_*; reflective
 * boundaries must be planes.  *id receives the surface index. */
int mcgb_add_surface(mcgb_ctx *ctx, int type, const double coef[4], int bc, int *id);
/* A cell is the intersection of n half-spaces (surf[k], sense[k] = +1 where
 * f > 0, -1 where f < 0) in `universe` (0 = root).  fill_kind
 * MCGB_FILL_MATERIAL: fill is a material index; MCGB_FILL_LATTICE: fill is a
 * lattice index (root-universe cells only).  Cells of a universe must
 * partition the space they cover. */
int mcgb_add_cell(mcgb_ctx *ctx, int universe, int n, const int *surf, const int *sense,
                  int fill_kind, int fill, int *id);
/* Rectangular x-y lattice with lower-left corner (x0, y0), square pitch,
 * nx * ny universes, element (ix, iy) at universes[ix + nx * iy].  Universe
 * cells are placed in element-centred coordinates. */
int mcgb_add_lattice(mcgb_ctx *ctx, double x0, double y0, double pitch, int nx, int ny,
                     const int *universes, int *id);

/* --------------------------------------------------------------------------- */
/* materials (Sec. 1: multigroup and continuous-energy physics)                  */
int mcgb_set_groups(mcgb_ctx *ctx, int G);
/* Multigroup material: sigma_t[G], sigma_s[G*G] as [from][to], nu_sigma_f[G],
 * chi[G] (any non-negative weights).  Row sums of sigma_s may not exceed sigma_t. */
int mcgb_add_material_mg(mcgb_ctx *ctx, const double *sigma_t, const double *sigma_s,
                         const double *nu_sigma_f, const double *chi, int *id);
/* Replace the cross sections of multigroup material id (same layout). */
int mcgb_update_material_mg(mcgb_ctx *ctx, int id, const double *sigma_t,
                            const double *sigma_s, const double *nu_sigma_f, const double *chi);
/* Pointwise nuclide: mass ratio A, n increasing energies E (eV) with elastic,
 * capture and fission cross sections (barns), mean neutrons per fission nu. */
int mcgb_add_nuclide_ce(mcgb_ctx *ctx, double A, int n, const double *E, const double *sig_s,
                        const double *sig_c, const double *sig_f, double nu, int *id);
/* Continuous-energy material: n nuclide ids with atom densities (atoms/b-cm). */
int mcgb_add_material_ce(mcgb_ctx *ctx, int n, const int *nuclides, const double *density,
                         int *id);

/* --------------------------------------------------------------------------- */
/* source and tallies                                                           */
/* kind MCGB_SRC_BOX: params {xmin,xmax,ymin,ymax,zmin,zmax}, positions uniform,
 * rejected until `accept` holds; MCGB_SRC_POINT: params {x,y,z}.
 * energy_kind CHI (group from chi of the located material), PDF (group weights
 * energy[0..n_energy)), FIXED (energy[0] eV), MAXWELL (fission spectrum).
 * dir_kind ISO or BEAM (unit vector beam[3]). */
int mcgb_set_source(mcgb_ctx *ctx, int kind, const double *params, int accept, int energy_kind,
                    const double *energy, int n_energy, int dir_kind, const double *beam);
/* Track-length flux tally.  filter: CELL (innermost cell), LATTICE (element
 * ix + nx iy of lattice 0), MATERIAL.  Energy bins: the groups (multigroup) or
 * n_edges increasing edges in eV (continuous energy). */
int mcgb_add_tally(mcgb_ctx *ctx, int filter, int n_edges, const double *edges, int *id);
/* End each history at its max_collisions-th collision (0 = no limit). */
int mcgb_set_max_collisions(mcgb_ctx *ctx, int max_collisions);
/* Time dependence (Sec. 1: time-dependent transport; Sec. 4 runs its
 * continuous-energy pin cell as a time-dependent fixed-source problem).  Source
 * particles start at time t0 (s); a flight ends where the particle's clock
 * reaches t_cut, at the distance (t_cut - t) / (1/v) when that is shorter than
 * the distances to collision and to the nearest surface (a tie goes to the
 * collision or crossing), and the history ends with fate 5.  Fission sites keep
 * the time of their collision.  Speeds: 1/v per group (s/cm, multigroup, set
 * with mcgb_set_inverse_speeds) or v = K sqrt(E / 1 eV), K = sqrt(2 e / m_n) *
 * 100 cm/s (continuous energy).  Fixed-source runs only (an eigenvalue run or
 * a derivative run fails); requires 0 <= t0 < t_cut < inf. */
int mcgb_set_time(mcgb_ctx *ctx, double t0, double t_cut);
/* Free-gas elastic scattering with a constant cross section (the model Sec. 4
 * assumes for its continuous-energy pin cell): below cut * kT (cut 0: 400) a
 * continuous-energy elastic collision samples the target's velocity from a
 * Maxwellian at temperature kT (eV) weighted by the relative speed and scatters
 * isotropically in the centre-of-mass frame; above it the target is at rest.
 * kT > 0 and finite, cut >= 0. */
int mcgb_set_free_gas(mcgb_ctx *ctx, double kT, double cut);
/* inv_v[G]: 1/v of each group in s/cm, positive and finite. */
int mcgb_set_inverse_speeds(mcgb_ctx *ctx, int G, const double *inv_v);
/* Time bins of a tally: n_edges increasing edges (s, first >= 0).  The tally
 * then scores, for every flight and bin, the time the flight spends in the bin
 * times 1 / (bin width): the mean neutron population per source particle in
 * the bin, per spatial bin and group or energy bin. */
int mcgb_set_tally_time_bins(mcgb_ctx *ctx, int tally, int n_edges, const double *edges);

/* --------------------------------------------------------------------------- */
/* runs                                                                         */
/* k-eigenvalue power iteration (Sec. 4): n histories per cycle, `inactive`
 * cycles discarded, statistics over `active` cycles. */
int mcgb_run_eigenvalue(mcgb_ctx *ctx, int64_t n, int inactive, int active, uint64_t seed);
/* The same power iteration in steps: begin (uploads the problem, allocates),
 * run n_cycles further cycles (any number of calls), finish (statistics).
 * mcgb_run_eigenvalue = begin + all cycles + finish. */
int mcgb_eigen_begin(mcgb_ctx *ctx, int64_t n, int inactive, int active, uint64_t seed);
int mcgb_eigen_cycles(mcgb_ctx *ctx, int n_cycles);
int mcgb_eigen_finish(mcgb_ctx *ctx);
/* Checkpoint and restart of a power iteration (no counterpart in the paper).
 * Between cycles of a run begun with mcgb_eigen_begin -- at least one cycle
 * run and at least one left -- mcgb_eigen_checkpoint writes into the host
 * buffer buf[0..cap) all that the remaining cycles and the final statistics
 * depend on: the run's sizes and seed, a fingerprint of the uploaded problem,
 * the cycle index, the per-cycle k sums, bank sizes and times so far, the
 * tally sums and sums of squares, the event counters, and the next cycle's
 * n sources as 64-byte mcgb_site records; a checksum ends it.  *needed = its
 * size (buf NULL: size query only; cap too small: MCGB_E_INVALID_ARG).  The
 * run goes on unchanged.
 * mcgb_eigen_restore begins the run again from such a record, on a context
 * holding the same problem (any mode or launch options; another fingerprint,
 * a bad checksum or a truncated record: MCGB_E_INVALID_ARG): the remaining
 * mcgb_eigen_cycles and mcgb_eigen_finish then give the results of the
 * uninterrupted run bit for bit, since every history's random stream depends
 * only on the seed, the cycle and its source index. */
int mcgb_eigen_checkpoint(mcgb_ctx *ctx, void *buf, size_t cap, size_t *needed);
int mcgb_eigen_restore(mcgb_ctx *ctx, const void *buf, size_t size);
/* Device time of each cycle (CUDA events on the context's stream): the
 * transport phase and the whole cycle, in ms. */
int mcgb_get_cycle_times(mcgb_ctx *ctx, int n_cycles, double *transport_ms, double *cycle_ms);
/* Fixed source: n source histories in `batches` statistical batches; fission
 * secondaries run as further generations until none remain. */
int mcgb_run_fixed_source(mcgb_ctx *ctx, int64_t n, int batches, uint64_t seed);

/* --------------------------------------------------------------------------- */
/* sharded power iteration (one rank of a multi-GPU run; Sec. 1 runs MC/DC     */
/* with MPI domain replication, here every cycle's histories are partitioned)  */
/* A fission site as exchanged between ranks: position, time, cell path,
 * material, child index and the global source index of its parent. */
typedef struct {
    double x, y, z, t;
    int32_t cell, ix, iy, ucell, mat, child;
    int64_t parent;
} mcgb_site;
/* One rank's share of an N-history k-eigenvalue power iteration of
 * inactive + active cycles: this context transports source indices
 * [j0, j0 + n) of every cycle (random streams cycle 2^32 + j as in a
 * single-device run).  Every cycle is three calls, in order:
 *   mcgb_shard_cycle   transport the slice; *m = sites the rank banked;
 *   mcgb_shard_export  write the rank's sites in (parent, child) order and its
 *                      sums [k_tl, k_c, tally sums (layout of mcgb_get_tally,
 *                      before division by N)] to caller device buffers;
 *   (the caller sums the sums over ranks and concatenates the ranks' sites in
 *    rank order -- the global (parent, child)-ordered bank -- moving bytes
 *    only)
 *   mcgb_shard_import  fold the all-rank sums into the run's statistics and
 *                      resample this rank's sources of the next cycle from the
 *                      global bank: source j takes site floor((j + xi) M / N),
 *                      at most M - 1, xi the cycle's draw -- exactly what one
 *                      device does, so the ranks together reproduce the
 *                      single-device run.
 * mcgb_shard_finish after the last cycle makes k, per-cycle k and bank sizes
 * and the tallies available through mcgb_get_k / mcgb_get_cycle_k /
 * mcgb_get_tally, as after mcgb_run_eigenvalue.  Every pointer of export and
 * import is a device pointer on the context's device, used in order on its
 * stream.  Calls out of order fail with MCGB_E_STATE; an empty global bank
 * fails import with MCGB_E_STATE.  Time-dependent problems are rejected. */
int mcgb_shard_begin(mcgb_ctx *ctx, int64_t N, int64_t j0, int64_t n, int inactive, int active,
                     uint64_t seed);
int mcgb_shard_cycle(mcgb_ctx *ctx, int cycle, int64_t *m);
/* bank_cap >= *m sites, sums_cap >= *n_sums; bank and sums NULL: only *n_sums */
int mcgb_shard_export(mcgb_ctx *ctx, mcgb_site *bank, size_t bank_cap, double *sums,
                      size_t sums_cap, size_t *n_sums);
/* sums: the all-rank sums; bank[0..M): the global ordered bank */
int mcgb_shard_import(mcgb_ctx *ctx, int cycle, const double *sums, const mcgb_site *bank,
                      int64_t M);
int mcgb_shard_finish(mcgb_ctx *ctx);

/* --------------------------------------------------------------------------- */
/* spatial domain decomposition (one rank of a multi-GPU run; Sec. 1: MC/DC's  */
/* domain "replicated or decomposed" over MPI)                                 */
/* A particle in flight between the domains of two ranks. */
typedef struct {
    double x, y, z, u, v, w, E;
    double drem;            /* remaining distance to the collision sampled before the
                               domain boundary cut the flight (< 0: none) */
    uint64_t s;             /* random-number state */
    int64_t hist;           /* the history's source index in its cycle */
    int32_t g, cell, ix, iy, ucell, mat, prob, root, nfis, ncoll, ncross, dest;
} mcgb_flight;
/* This context owns the slab cuts[rank] <= coordinate `axis` (0 x, 1 y, 2 z)
 * < cuts[rank + 1] of an N-history k-eigenvalue power iteration of inactive +
 * active cycles (cuts: n_domains + 1 increasing values, +-inf allowed at the
 * ends).  A history is transported by the rank whose slab holds it: a flight
 * that reaches the slab's boundary stops there and the particle -- with the
 * rest of its sampled collision distance, so no random number is drawn again
 * -- is handed to the neighbouring rank.  Random streams are per history, so
 * every history is the single-device one up to the rounding of the cut
 * flights (one domain: identical).  Every cycle, in order:
 *   mcgb_domain_sources  the cycle's sources in this slab (cycle 0: sampled
 *                        from the source definition; later: resampled from
 *                        the global ordered bank of the previous cycle,
 *                        bank[0..M), device records);
 *   repeat:  mcgb_domain_sweep (transport every particle in the slab until it
 *            dies or leaves; *n_out = particles leaving), mcgb_domain_outbox
 *            (copy them to a device buffer), and mcgb_domain_inbox with the
 *            outboxes of all ranks (each rank keeps the particles addressed
 *            to it) -- until no rank has a particle leaving;
 *   mcgb_domain_export   the rank's share of the cycle end, to device buffers:
 *                        nfis[N] = sites banked by each history that ended in
 *                        this slab (0 for the others), sites[0..m) = the sites
 *                        banked in this slab (any order), sums = [k_tl, k_c,
 *                        tally sums]; *m, *n_sums their sizes (sites and sums
 *                        NULL: only the sizes);
 *   mcgb_domain_import   the all-rank sums, nfis summed over ranks, and every
 *                        rank's sites (concatenated, any order): the statistics
 *                        of the cycle and the global (parent, child)-ordered bank.
 * mcgb_domain_finish then fills mcgb_get_k / mcgb_get_cycle_k / mcgb_get_tally
 * as mcgb_run_eigenvalue does.  mcgb_domain_records writes, for checks, the
 * per-history records of the last cycle's histories that ended in this slab
 * (device arrays of N; zero for the others, so that their sum over ranks is
 * the complete record).  All arrays of these calls are device pointers on the
 * context's device, used in order on its stream.  Out-of-order calls fail with
 * MCGB_E_STATE; time-dependent problems are rejected. */
int mcgb_domain_begin(mcgb_ctx *ctx, int64_t N, int inactive, int active, uint64_t seed, int axis,
                      const double *cuts, int n_domains, int rank);
int mcgb_domain_sources(mcgb_ctx *ctx, int cycle, const mcgb_site *bank, int64_t M);
int mcgb_domain_sweep(mcgb_ctx *ctx, int64_t *n_out);
int mcgb_domain_outbox(mcgb_ctx *ctx, mcgb_flight *out, size_t cap);
int mcgb_domain_inbox(mcgb_ctx *ctx, const mcgb_flight *in, int64_t n);
int mcgb_domain_export(mcgb_ctx *ctx, int32_t *nfis, mcgb_site *sites, size_t sites_cap,
                       double *sums, size_t sums_cap, size_t *m, size_t *n_sums);
int mcgb_domain_import(mcgb_ctx *ctx, int cycle, const double *sums, const int32_t *nfis,
                       const mcgb_site *sites, int64_t M);
int mcgb_domain_finish(mcgb_ctx *ctx);
int mcgb_domain_records(mcgb_ctx *ctx, int32_t *n_coll, int32_t *n_cross, int32_t *n_fis,
                        int32_t *fate, int32_t *g_end, uint64_t *rng_end);

/* --------------------------------------------------------------------------- */
/* results                                                                      */
/* out[6] = k (track length) mean, sd; k (collision) mean, sd; k (analog) mean, sd. */
int mcgb_get_k(mcgb_ctx *ctx, double out[6]);
/* Per-cycle k (track length), k (collision) and bank size, n_cycles entries. */
int mcgb_get_cycle_k(mcgb_ctx *ctx, int n_cycles, double *k_tl, double *k_col, int64_t *bank);
/* bins, energy bins (groups) and time bins (1 without time bins) of a tally */
int mcgb_tally_size(mcgb_ctx *ctx, int tally, int *n_bins, int *n_ebins, int *n_tbins);
/* mean and sd per source particle, [bin][ebin][tbin], cap elements each. */
int mcgb_get_tally(mcgb_ctx *ctx, int tally, double *mean, double *sd, size_t cap,
                   size_t *needed);
int mcgb_get_counters(mcgb_ctx *ctx, mcgb_counters *out);
/* One-kernel-per-event mode (Sec. 2's event-based form): device time summed
 * over the first flight launch of every generation run so far (one k_advance
 * over the whole generation, identity list), the particles those launches
 * processed, their number, and the algorithmic state bytes one particle moves
 * in such a launch (fields loaded and stored, queue entry).  Zeros until an
 * event-mode generation has run.  Any output pointer may be NULL. */
int mcgb_get_event_timing(mcgb_ctx *ctx, double *advance_ms, int64_t *particles, int64_t *launches,
                          double *bytes_per_particle);

/* Per-history records (opts.record_histories): last cycle (eigenvalue) or
 * generation 0 (fixed source).  fate: 0 absorbed, 1 leaked, 2 cut by
 * max_collisions, 3 lost, 4 event cap, 5 reached the time cutoff.  Arrays of
 * cap elements. */
int mcgb_get_histories(mcgb_ctx *ctx, size_t cap, int32_t *n_coll, int32_t *n_cross,
                       uint64_t *rng_end, int32_t *n_fis, int32_t *fate, int32_t *g_end,
                       size_t *needed);
/* Fission bank of the last cycle (eigenvalue) or generation 0 (fixed source),
 * in (parent, child) order: xyz[3*cap], parent[cap], child[cap], mat[cap]. */
int mcgb_get_bank(mcgb_ctx *ctx, size_t cap, double *xyz, int64_t *parent, int32_t *child,
                  int32_t *mat, size_t *needed);

/* --------------------------------------------------------------------------- */
/* derivatives (likelihood ratio with replay; the paper has no counterpart)    */
/* Forward: fixed-source run of n histories (1 batch) that keeps what the replay
 * needs: per-particle detector tallies and every generation's sorted bank.
 * tally_out[G] = the detector cell's track-length tally per group per source. */
int mcgb_forward_fixed(mcgb_ctx *ctx, int64_t n, uint64_t seed, int det_cell, double *tally_out);
/* Backward: replays every history of the last forward run from its random
 * stream and accumulates score x downstream-tally for T = sum_g w[g] T_g:
 * d_sigt[m*G+g], d_sigs[(m*G+g)*G+g'], d_nusf[m*G+g] per source particle.
 * Parameters equal to 0 take no score. */
int mcgb_backward_fixed(mcgb_ctx *ctx, const double *weights, double *d_sigt, double *d_sigs,
                        double *d_nusf);

/* Device-pointer variants of the three calls above, for callers whose arrays
 * live on the context's device (the torch binding): every array argument is a
 * device pointer on the context's device, caller-owned, read or written in
 * order on the context's stream; no array goes through host memory.
 *
 * mcgb_update_material_mg_dev: new Sigma_t [n_mat][G], Sigma_s [n_mat][G][G]
 *   ([from][to]) and nuSigma_f [n_mat][G] of materials first .. first+n_mat-1
 *   (chi unchanged), written into the device tables (the world is built from
 *   the definition first if it is not current).  The host-side definition
 *   keeps its old values: a later definition change or a host-array run
 *   rebuilds the tables from it.  Values are checked on the device; a
 *   negative value or Sigma_s,tot > Sigma_t leaves that row unchanged and
 *   makes the next mcgb_forward_fixed_dev fail with MCGB_E_INVALID_ARG.
 * mcgb_forward_fixed_dev: as mcgb_forward_fixed on the current device tables;
 *   tally[G] (device) may be NULL.  The run's control flow still reads bank
 *   sizes and status flags on the host.
 * mcgb_backward_fixed_dev: as mcgb_backward_fixed with weights[G],
 *   d_sigt[M*G], d_sigs[M*G*G], d_nusf[M*G] on the device; returns when the
 *   results are written. */
int mcgb_update_material_mg_dev(mcgb_ctx *ctx, int first, int n_mat, const double *sigma_t,
                                const double *sigma_s, const double *nu_sigma_f);
int mcgb_forward_fixed_dev(mcgb_ctx *ctx, int64_t n, uint64_t seed, int det_cell, double *tally);
int mcgb_backward_fixed_dev(mcgb_ctx *ctx, const double *weights, double *d_sigt, double *d_sigs,
                            double *d_nusf);

/* --------------------------------------------------------------------------- */
/* batching: many independent fixed-source problems in one persistent launch    */
int mcgb_batch_create(mcgb_batch **out, const mcgb_opts *opts);
int mcgb_batch_destroy(mcgb_batch *b);
/* Add a problem defined in `problem` (its tables are copied; the context may be
 * destroyed afterwards): n source histories in `batches` batches, seed. */
int mcgb_batch_add_problem(mcgb_batch *b, mcgb_ctx *problem, int64_t n, int batches,
                           uint64_t seed, int *id);
/* Time candidate launch shapes on a fraction of the work, time the three
 * fastest again on the whole batch, and return the best (the budget bounds
 * the first stage); results are cached per (problem signature, device) in
 * memory and, when the environment variable MCGB_TUNE_CACHE names a file, on
 * disk. */
int mcgb_batch_autotune(mcgb_batch *b, int budget_ms, mcgb_tune *out);
/* Run every problem: tune NULL = the cached or default shape. */
int mcgb_batch_run(mcgb_batch *b, const mcgb_tune *tune);
int mcgb_batch_tally(mcgb_batch *b, int problem, int tally, double *mean, double *sd,
                     size_t cap, size_t *needed);
int mcgb_batch_counters(mcgb_batch *b, mcgb_counters *out);

/* --------------------------------------------------------------------------- */
/* building blocks on the device, for checks against other implementations     */
/* out[i*n_draws + k] = k-th state of stream first_id + i of `seed` (63-bit LCG,
 * stride 152917; Sec. 1's replicable random numbers). */
int mcgb_rng_states(mcgb_ctx *ctx, uint64_t seed, uint64_t first_id, int64_t n_streams,
                    int n_draws, uint64_t *out);
/* out[i] = ln(xi[i]) for xi[i] = k 2^-53, k in [1, 2^53] (the transport's log). */
int mcgb_log(mcgb_ctx *ctx, int64_t n, const double *xi, double *out);
/* The transport's float64 square root, quotient and reciprocal, which it
 * computes on the integer and float32 pipes (the paper prescribes none): for
 * each i, out[3*i] = sqrt(a[i]), out[3*i+1] = a[i] / b[i], out[3*i+2] =
 * 1 / b[i], each the IEEE round-to-nearest value (a negative a[i] gives NaN).
 * a, b: n host doubles each; out: 3 n host doubles. */
int mcgb_fpint_ops(mcgb_ctx *ctx, int64_t n, const double *a, const double *b, double *out);
/* FP64 throughput of this device, measured: a grid of 8 blocks of 256 threads
 * per SM runs independent fused multiply-add chains, `iters` steps of 8 chains
 * per thread, timed with CUDA events on the context's stream after one
 * untimed launch.  *ops_per_s = FP64 thread-instructions per second (an FMA
 * counts once), *ms = the timed launch.  The roofline of the FP64-bound
 * transport kernels is taken against this (the paper gives no peak). */
int mcgb_fp64_throughput(mcgb_ctx *ctx, int64_t iters, double *ops_per_s, double *ms);
/* Geometry probe: locate each point (direction dir) and the distance to the
 * nearest boundary.  path[5*i..] = root cell, ix, iy, universe cell, material. */
int mcgb_probe(mcgb_ctx *ctx, int64_t n, const double *pos, const double *dir, int32_t *path,
               double *dist, int32_t *kind);
/* Continuous-energy lookup of material `mat` at n energies: out[4*i..] =
 * Sigma_t, nuSigma_f, Sigma_s, Sigma_f. */
int mcgb_ce_lookup(mcgb_ctx *ctx, int mat, int64_t n, const double *E, double *out);

/* --------------------------------------------------------------------------- */
/* allocation-free bank ordering (the paper has no counterpart)                 */
/* For callers that cannot give the library device memory: their GPU memory is
 * owned by another allocator (for example a framework's caching allocator that
 * has reserved the device), or they must not allocate once running.  Given
 * n_fis[n], the fission sites each history of a cycle banked (device pointer),
 * writes first[j] = sites banked by histories 0..j-1 -- the position of history
 * j's first site in the (parent, child) ordered bank -- and *total = all sites
 * (device pointers), on cuda_stream (NULL = legacy default stream), with the
 * same kernels as the library's own cycle end.  It allocates nothing: its
 * scratch is a 16 KiB array built into the library, held on every GPU that
 * loads it until the process exits.  n may be at most 16777216; larger n is
 * rejected with MCGB_E_INVALID_ARG.  The first call on a device (make it the
 * current device) looks up the array's device address; make that first call
 * before any stream capture.  Each device holds its own copy of the array, and
 * all calls on one device share it: calls that overlap on the same GPU (on
 * concurrent streams) race, so order them on one stream; calls on different
 * devices do not interfere.  Nothing in the array needs clearing between calls.
 * Returns MCGB_OK or MCGB_E_INVALID_ARG / MCGB_E_CUDA. */
int mcgb_bank_offsets_noalloc(const int32_t *n_fis, int64_t n, int32_t *first, int32_t *total,
                              void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MCGB_H */
