// world.h -- device-resident problem tables, particle state and run buffers.
//
// Layout (all in HBM, one allocation per array):
//  * World: every table of every problem of a run, concatenated with global
//    indices (a single problem is a batch of one).  Read-only during a run.
//  * Particles: structure-of-arrays state of the particles in flight (one
//    slot per history of the current cycle or generation).
//  * Bank: structure-of-arrays fission sites appended during a cycle, put in
//    (parent, child) order afterwards through a permutation.
#pragma once
#include <cstdint>

namespace mcgb {

constexpr int MAX_EVENTS = 1000000;   // events per history before it is cut
constexpr int MAX_TRIES = 10000;      // source rejection attempts
constexpr int MAX_NUC = 8;            // nuclides per continuous-energy material
constexpr int MAX_G = 16;             // groups per multigroup problem
constexpr double E_MIN = 1.0e-5;      // eV
constexpr double E_MAX = 2.0e7;       // eV
constexpr double MAXWELL_T = 1.33e6;  // eV
constexpr int KSLOTS = 4096;          // spread accumulators for k estimators

enum { SURF_PX = 0, SURF_PY = 1, SURF_PZ = 2, SURF_PLANE = 3, SURF_CYLZ = 4, SURF_SPHERE = 5 };
enum { BC_NONE = 0, BC_VACUUM = 1, BC_REFLECT = 2 };
enum { FILL_MAT = 0, FILL_LAT = 1 };
enum { SRC_BOX = 0, SRC_POINT = 1 };
enum { E_CHI = 0, E_PDF = 1, E_FIXED = 2, E_MAXWELL = 3 };
enum { DIR_ISO = 0, DIR_BEAM = 1 };
enum { FILTER_CELL = 0, FILTER_LATTICE = 1, FILTER_MATERIAL = 2 };
// boundary kinds found by the distance search, in precedence order
enum { B_NONE = 0, B_ROOT = 1, B_LATX = 2, B_LATY = 3, B_UNIV = 4 };
// history fates
enum { FATE_ALIVE = -1, FATE_ABSORBED = 0, FATE_LEAKED = 1, FATE_CUT = 2, FATE_LOST = 3,
       FATE_CAPPED = 4, FATE_TIME = 5,
       // domain decomposition: left this rank's slab / never in it this cycle
       FATE_MOVED = 6, FATE_ELSEWHERE = 7 };
// error flags raised by kernels
enum { ERR_BANK_OVERFLOW = 1, ERR_SOURCE = 2, ERR_QUEUE = 4, ERR_ITER = 8 };

struct ProblemDev {
    int cell0, mat0;      // first global cell / material id of the problem (tally bins are local)
    int root_univ;        // global universe id of the problem's root
    int lattice0;         // global id of its first lattice (lattice filter), -1 if none
    int ce;               // continuous energy
    int G;                // groups (multigroup)
    int src_kind, src_accept, src_ekind, src_dkind;
    double src_p[6];
    double src_beam[3];
    double src_E;
    int src_cdf_off, src_ncdf;
    int tally_first, tally_count;
    int max_coll;
    int batches;
    uint64_t seed;
    int64_t n;            // source histories
    // time dependence (fixed source): births at t0, flights cut at tcut; 1/v per
    // group from g_invv[invv_off + g] (multigroup) or 1 / (kv sqrt(E)) (CE)
    int time_on;
    int invv_off;
    double t0, tcut;
    // free-gas elastic scattering below fg_emax (fg_kT > 0 enables it)
    double fg_kT, fg_emax, fg_ikT;   // fg_ikT = 1 / fg_kT, rounded once
};

struct World {
    int nprob;
    int need_iw;            // some z-plane exists: 1/w is read (else it is never computed)
    const ProblemDev *prob;
    // surfaces
    const int *s_type, *s_bc;
    const double *s_coef;   // 4 per surface
    const double *s_r2;     // R*R for quadrics
    const int *s_zc;        // z-cylinder centred at (+0, +0)
    // cells and half-spaces
    const int *c_univ, *c_off, *c_nhs, *c_fillk, *c_fill;
    const int *hs_surf, *hs_sense;
    const int *hs_coff, *hs_cand;   // candidate cells across each half-space (CSR)
    const int *u_off, *u_cells;     // cells of each universe (CSR, definition order)
    const int *u_edge;              // cell holding a lattice element's whole boundary, or -1
    const int *c_skiproot;          // lattice root cell whose planes interior elements never reach first
    const int *hs_side;             // per half-space of such a cell: lattice side of its plane (1..4)
    const int *c_inner;             // universe cell inside a surface strictly inside its element
    const int *c_rootfar;           // lattice root cell whose surfaces are planes on or beyond the lattice's edges
    // lattices; wall and centre coordinates are precomputed with the same
    // expressions the transport would evaluate: x0 + (double)i * pitch and
    // x0 + ((double)i + 0.5) * pitch (bit-identical, fewer FP64 instructions)
    const double *l_x0, *l_y0, *l_pitch;
    const int *l_nx, *l_ny, *l_uoff, *l_univ;
    const int *l_woff;              // first wall entry of each lattice: nx + 1 x walls, then ny + 1 y walls
    const double *l_wall, *l_ctr;   // per lattice: x walls, y walls; x centres, y centres (same offsets)
    // multigroup materials (per-material group count and offsets)
    const int *m_G, *m_goff, *m_ggoff, *m_fissile;
    const double *g_sigt, *g_mfp, *g_nusf, *g_mu, *g_mufl, *g_mufr, *g_ps, *g_stot, *g_chicdf;
    const double *gg_sigs, *gg_scdf;
    // continuous energy
    int nunion, nnuc;
    const double *Eu;        // union grid
    // union-grid buckets: key = (bits of E >> 44) - ukey0 clamped to [0, nukey);
    // ukey_lo[b] = search result at the lower edge of bucket b (nukey + 1 entries)
    long long ukey0;
    int nukey;
    const int *ukey_lo;
    // macroscopic flight cross sections per CE material on its own union grid:
    // points cm_E[cm_off[m] + k], records of 6 doubles (E_k, 1/dE_k, St_k, dSt_k,
    // Sf_k, dSf_k), bucket index cm_klo[cm_koff[m] + b] keyed from cm_key0[m]
    const int *cm_off, *cm_n, *cm_nkey, *cm_koff, *cm_klo;
    const long long *cm_key0;
    const double *cm_E, *cm_rec;
    const int *umap;         // [nuc * nunion + k]: nuclide interval of union interval k
    const int *n_ivoff;      // first interval of each nuclide
    const double *n_iv;      // 8 doubles per interval: E, 1/dE, s, ds, c, dc, f, df
    const double *n_A, *n_nu;
    const double *n_kin;      // per nuclide {A, 2A, A^2 + 1, 1/(A + 1)^2, 1/(A + 1), 1/A} (kinematics)
    const int *mc_off, *mc_n, *mc_nuc, *mc_fissile;
    const double *mc_dens;
    // source group distributions
    const double *src_cdf;
    // log tables: ln(1 + j/256), 1/(1 + j/256), (e - 53) ln 2
    const int64_t *lnc_q, *eln2_q;   // ln(1 + j/256) and (e - 53) ln 2 in Q57
    const uint64_t *invc_q;          // 256 / (256 + j) in Q63, rounded down
    // tallies (global tally ids; accumulators [rep][acc_size]); a tally with
    // t_ntb > 0 time bins has edges t_tedges[t_toff + k] and 1 / width
    // t_tinvw[t_toff + k] and scores population instead of track length
    const int *t_filter, *t_nbins, *t_ne, *t_off, *t_eoff, *t_nedges, *t_batches;
    const double *t_edges;
    const int *t_ntb, *t_toff;
    const double *t_tedges, *t_tinvw;
    int acc_size, nrep;
    // time dependence: inverse group speeds; CE speed constant v = kv sqrt(E);
    // time_any: some problem is time dependent or some tally has time bins (the
    // persistent kernels are then launched in their time-aware instantiation)
    const double *g_invv;
    double kv;
    int time_any;
    int ce_any;             // some problem has continuous-energy physics (particles carry E)
};

struct Particles {
    double *x, *y, *z, *u, *v, *w, *E, *t;
    double *iu, *iv, *iw;   // direction reciprocals
    double *kt, *kc;      // per-history k estimator sums (track length, collision)
    double *drem;         // domain decomposition: rest of a cut flight's collision distance
    uint64_t *s;
    int *g, *cell, *ix, *iy, *ucell, *mat, *uk, *prob, *root, *nfis, *ncoll, *ncross, *bwhich;
    signed char *bkind, *fate;
    int64_t cap;
};

struct Bank {
    double *x, *y, *z, *t;
    int *cell, *ix, *iy, *ucell, *mat, *parent, *child, *root, *prob;
    int64_t cap;
};

// The slab a rank owns in a spatially decomposed run: lo <= coordinate `axis`
// (0 x, 1 y, 2 z) < hi; the outermost slabs reach to -inf and +inf.
struct DomainCut {
    int axis;
    double lo, hi;
};

// One fission-bank site as exchanged between the ranks of a sharded run (the
// layout of the C ABI's mcgb_site: 64 bytes).
struct ShardSite {
    double x, y, z, t;
    int32_t cell, ix, iy, ucell, mat, child;
    int64_t parent;
};
static_assert(sizeof(ShardSite) == 64, "site records are 64 bytes");

// A particle handed between the ranks of a spatially decomposed run (the
// layout of the C ABI's mcgb_flight: 128 bytes).
struct FlightRec {
    double x, y, z, u, v, w, E, drem;
    uint64_t s;
    int64_t hist;
    int32_t g, cell, ix, iy, ucell, mat, prob, root, nfis, ncoll, ncross, dest;
};
static_assert(sizeof(FlightRec) == 128, "flight records are 128 bytes");

// Per-run device counters and accumulators.
struct RunBufs {
    double *kacc;          // [KSLOTS][2]: track-length and collision k sums
    double *tacc;          // tally accumulators [nrep][acc_size]
    int *bank_n;           // fission sites appended this cycle
    int *err;              // ERR_* flags
    int *q_n;              // queue lengths: [0] cross, [1] collide, [2] next active
    double *own;           // derivative mode: per-slot detector tally by group (or null)
    int own_cell, own_G;
};

}  // namespace mcgb
