// host_world.h -- host-side problem definitions and their flattening into the
// device tables of world.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "world.h"

namespace mcgb {

struct CellDef {
    int univ, fillk, fill;
    std::vector<int> surf, sense;
};
struct LatDef {
    double x0, y0, pitch;
    int nx, ny;
    std::vector<int> univ;
};
struct MatMGDef {
    std::vector<double> sigt, sigs, nusf, chi;
};
struct NucDef {
    double A, nu;
    std::vector<double> E, s, c, f;
};
struct MatCEDef {
    std::vector<int> nuc;
    std::vector<double> dens;
};
struct SrcDef {
    int kind = -1, accept = 0, ekind = 0, dkind = 0;
    double p[6] = {0, 0, 0, 0, 0, 0};
    double beam[3] = {0, 0, 1};
    double E = 0.0;
    std::vector<double> pdf;
};
struct TallyDef {
    int filter;
    std::vector<double> edges;
    std::vector<double> tedges;   // time bin edges (empty: no time bins)
};

// Everything a user defines for one problem through the C ABI.
struct ProblemDef {
    int G = 0;
    int ce = -1;   // -1 undecided, 0 multigroup, 1 continuous energy
    std::vector<int> s_type, s_bc;
    std::vector<double> s_coef;
    std::vector<CellDef> cells;
    std::vector<LatDef> lats;
    std::vector<MatMGDef> mg;
    std::vector<NucDef> nucs;
    std::vector<MatCEDef> mce;
    SrcDef src;
    std::vector<TallyDef> tallies;
    int max_coll = 0;
    bool time_on = false;
    double t0 = 0.0, tcut = 0.0;
    std::vector<double> invv;    // inverse group speeds (multigroup)
    double fg_kT = 0.0, fg_cut = 0.0;   // free gas: kT (eV), applied below fg_cut * kT
    std::string check() const;   // empty when runnable
};

// Run parameters of one problem inside a flattened world.
struct ProblemRun {
    const ProblemDef *def;
    int64_t n;
    int batches;   // tally batches (1 for eigenvalue: cycles are the batches)
    uint64_t seed;
};

// Device copy of a flattened world.
struct DeviceWorld {
    World W{};
    void *arena = nullptr;
    size_t bytes = 0;
    std::vector<ProblemDev> probs;      // host copy
    std::vector<int> tally_first;       // global tally id of each problem's first tally
    std::vector<int> t_off, t_nbins, t_ne, t_batches, t_ntb;  // host copies per global tally
    int acc_size = 0, nrep = 1;
    uint64_t fingerprint = 0;           // FNV-1a of the uploaded bytes (checkpoints)
    ~DeviceWorld();
};

// Flatten problems and upload; returns an error message or "".
std::string build_world(const std::vector<ProblemRun> &runs, DeviceWorld &dw, cudaStream_t st);

// Host-side tables identical to the device ones (shared with the checks).
int64_t ln_table_q57(int j);
int64_t ln2_q57();
void make_cdf(const double *w, int n, double *cdf);

}  // namespace mcgb
