/*
 * mcoracle.h -- plain, slow, history-based CPU reference for Monte Carlo
 * neutral-particle transport (test infrastructure only).
 *
 * This is the oracle that the CUDA library is checked against.  Only the test
 * suite, the package's smoke check and the benchmark's CPU-baseline leg use it;
 * the library never calls, links or loads it.  It shares no source with the
 * CUDA path.
 *
 * Capabilities follow the paper's statement of what the transport code does
 * (Sec. 1: multigroup and continuous-energy physics, constructive solid
 * geometry with surface tracking, k-eigenvalue and fixed-source problems,
 * replicable random numbers).  The paper prints no formulas for any of these,
 * so each step follows the textbook algorithm; every choice the paper leaves
 * open is stated where the code makes it.
 *
 * Two arithmetic modes.  PLAIN (the default) evaluates every step as its
 * definition is written: ln from libm, distances by true division, no fused
 * multiply-adds, continuous-energy cross sections as the sum over nuclides of
 * N_i sigma_i(E), sampling against unnormalised partial sums.  STRICT follows
 * the rounding conventions the CUDA library chose for speed (a table-driven
 * logarithm, carried direction reciprocals, explicit fused multiply-adds,
 * per-material macroscopic tables), so that histories can be compared bit for
 * bit; every such convention is marked "Strict:" where it is made.  Both modes
 * take the same random draws in the same order.
 *
 * All functions return 0 on success or a negative code; orc_error() gives a
 * message.  Arrays passed in are copied.  Output arrays are caller-owned.
 */
#ifndef MCORACLE_H
#define MCORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_ctx orc_ctx;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ESTATE = -2, ORC_EOOM = -4, ORC_ELOST = -6,
       ORC_ETIMEOUT = -7 };
enum { ORC_PX = 0, ORC_PY = 1, ORC_PZ = 2, ORC_PLANE = 3, ORC_CYLZ = 4, ORC_SPHERE = 5 };
enum { ORC_BC_NONE = 0, ORC_BC_VACUUM = 1, ORC_BC_REFLECT = 2 };
enum { ORC_FILL_MATERIAL = 0, ORC_FILL_LATTICE = 1 };
enum { ORC_SRC_BOX = 0, ORC_SRC_POINT = 1 };
enum { ORC_ACCEPT_ANY = 0, ORC_ACCEPT_FISSILE = 1 };
enum { ORC_E_CHI = 0, ORC_E_PDF = 1, ORC_E_FIXED = 2, ORC_E_MAXWELL = 3 };
enum { ORC_DIR_ISO = 0, ORC_DIR_BEAM = 1 };
enum { ORC_FILTER_CELL = 0, ORC_FILTER_LATTICE = 1, ORC_FILTER_MATERIAL = 2 };

enum { ORC_PLAIN = 0, ORC_STRICT = 1 };

orc_ctx *orc_create(void);
void orc_destroy(orc_ctx *c);
const char *orc_error(const orc_ctx *c);
/* arithmetic mode of the context's runs (ORC_PLAIN, the default, or ORC_STRICT) */
int orc_set_arith(orc_ctx *c, int mode);

/* geometry */
int orc_add_surface(orc_ctx *c, int type, const double coef[4], int bc);
int orc_add_cell(orc_ctx *c, int universe, int n, const int *surf, const int *sense,
                 int fill_kind, int fill);
int orc_add_lattice(orc_ctx *c, double x0, double y0, double pitch, int nx, int ny,
                    const int *universes);
/* multigroup data: sigma_s is [from][to] */
int orc_set_groups(orc_ctx *c, int G);
int orc_add_material_mg(orc_ctx *c, const double *sigma_t, const double *sigma_s,
                        const double *nu_sigma_f, const double *chi);
/* continuous-energy data (energies in eV, cross sections in barns) */
int orc_add_nuclide(orc_ctx *c, double A, int n, const double *E, const double *sig_s,
                    const double *sig_c, const double *sig_f, double nu);
int orc_add_material_ce(orc_ctx *c, int n, const int *nuclides, const double *density);
/* source: box = {xmin,xmax,ymin,ymax,zmin,zmax}; point = {x,y,z} */
int orc_set_source(orc_ctx *c, int kind, const double *params, int accept, int energy_kind,
                   const double *energy, int n_energy, int dir_kind, const double *beam);
int orc_add_tally(orc_ctx *c, int filter, int n_edges, const double *edges);
int orc_set_max_collisions(orc_ctx *c, int max_collisions);

/* Time dependence (Sec. 1: time-dependent transport; Sec. 4 runs its pin cell
 * in time-dependent fixed-source mode).  Source particles start at t0; a flight
 * is cut where the particle's clock reaches t_cut (fate 5).  Multigroup speeds
 * are given as 1/v per group (s/cm); continuous energy uses v = K sqrt(E),
 * K = sqrt(2 e / m_n) * 100 cm/s per sqrt(eV).  Fixed-source runs only. */
int orc_set_time(orc_ctx *c, double t0, double t_cut);
/* Free-gas elastic scattering with a constant cross section (Sec. 4) for
 * continuous-energy collisions below cut * kT (cut 0: 400); kT in eV. */
int orc_set_free_gas(orc_ctx *c, double kT, double cut);
int orc_set_inverse_speeds(orc_ctx *c, int G, const double *inv_v);
/* time bins of a tally: it then scores, per bin, the time each particle spends
 * in the bin divided by the bin width (mean population per source particle) */
int orc_set_tally_time_bins(orc_ctx *c, int tally, int n_edges, const double *edges);

/* runs */
int orc_run_eigen(orc_ctx *c, int64_t n, int inactive, int active, uint64_t seed, int threads);
int orc_run_fixed(orc_ctx *c, int64_t n, int batches, uint64_t seed, int threads);

/* results */
int orc_get_k(const orc_ctx *c, double out[6]); /* k_TL mean, sd, k_C mean, sd, k_analog mean, sd */
int orc_get_cycle_k(const orc_ctx *c, int n_cycles, double *k_tl, double *k_c, int64_t *bank_size);
int orc_tally_size(const orc_ctx *c, int tally, int *n_bins, int *n_ebins, int *n_tbins);
int orc_get_tally(const orc_ctx *c, int tally, double *mean, double *sd);
/* counters: histories, collisions, crossings, leaks, lost, capped, generations,
 * time cuts */
int orc_get_counters(const orc_ctx *c, int64_t out[8]);
/* per-history record of the last cycle (eigen) or generation 0 (fixed):
 * fate 0 absorbed, 1 leaked, 2 cut by max_collisions, 3 lost, 4 event cap,
 * 5 reached the time cutoff */
int64_t orc_history_count(const orc_ctx *c);
int orc_get_histories(const orc_ctx *c, int32_t *n_coll, int32_t *n_cross, uint64_t *rng_end,
                      int32_t *n_fis, int32_t *fate, int32_t *g_end);
/* histories j = idx[k] of the first cycle / generation 0, each run alone */
int orc_histories_by_index(orc_ctx *c, uint64_t seed, int64_t n_idx, const int64_t *idx,
                           int32_t *n_coll, int32_t *n_cross, uint64_t *rng_end, int32_t *n_fis,
                           int32_t *fate, int32_t *g_end);
/* fission bank of the last cycle / generation 0, in (parent, child) order */
int64_t orc_bank_count(const orc_ctx *c);
int orc_get_bank(const orc_ctx *c, double *xyz, int64_t *parent, int32_t *child, int32_t *mat);

/* likelihood-ratio derivatives of one cell's track-length tally (fixed source,
 * multigroup).  weights[g] combines the per-group tallies into the scalar
 * T = sum_g weights[g] * T_g whose derivative is returned:
 * d_sigt[m*G+g], d_sigs[(m*G+g)*G+g'], d_nusf[m*G+g] (per source particle),
 * with tally[g] the detector tally means. */
int orc_grad_fixed(orc_ctx *c, int64_t n, uint64_t seed, int cell, const double *weights,
                   double *d_sigt, double *d_sigs, double *d_nusf, double *tally);

/* building blocks exposed for the pin tests; `mode` is ORC_PLAIN or ORC_STRICT */
uint64_t orc_rng_skip(uint64_t s, uint64_t n);
uint64_t orc_rng_stream(uint64_t seed, uint64_t id);
uint64_t orc_rng_next(uint64_t s);
double orc_rng_xi(uint64_t s);
/* ln xi by the strict mode's table-driven method (xi in (0, 1]) */
double orc_log(double xi);
/* entry j (0..255) of that method's table of ln(1 + j/256) */
int64_t orc_log_table_q57(int j);
/* index of the bank site that source j of N takes after a cycle banked M sites,
 * for the resampling draw xi = n 2^-53 (n in [1, 2^53]) */
int64_t orc_site_index(int64_t j, uint64_t n, int64_t M, int64_t N);
int orc_iso_dir(uint64_t *s, double out[3], int mode);
int orc_elastic(double E, double A, const double dir[3], uint64_t *s, double out[4], int mode);
int orc_free_gas(double E, double A, double kT, const double dir[3], uint64_t *s, double out[4],
                 int mode);
double orc_maxwell(uint64_t *s, int mode);
int orc_probe(orc_ctx *c, const double pos[3], const double dir[3], int out_path[5],
              double *dist, int *kind);
int orc_ce_lookup(orc_ctx *c, int material, double E, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
