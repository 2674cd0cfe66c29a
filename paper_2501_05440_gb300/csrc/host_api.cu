// host_api.cu -- the C ABI: problem definition, run drivers, results.
//
// A run keeps all particle state, banks and accumulators in device memory.
// Power iteration per cycle: transport N histories (event mode: a host loop of
// advance / cross / collide kernels over compacted queues; segment mode: a host
// loop of one monolithic segment kernel; persistent mode: one grid-resident
// kernel), then on the device: reduce k estimators, scan the
// per-history site counts, permute the bank into (parent, child) order,
// resample N sources, fold the cycle's tallies into the batch statistics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mcgb.h"
#include "host_world.h"
#include "kernels.h"
#include "transport.cuh"

using namespace mcgb;

static thread_local std::string g_err = "";

static int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

namespace mcgb {
// lets other translation units report through mcgb_last_error()
int set_error(int code, const char *msg) { return fail(code, msg); }
}  // namespace mcgb

#define CK(expr)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? MCGB_E_OOM : MCGB_E_CUDA,    \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));           \
    } while (0)

#define CKR(expr)                  \
    do {                           \
        int r_ = (expr);           \
        if (r_ != MCGB_OK) return r_; \
    } while (0)

// ---------------------------------------------------------------------------
// device buffers of a run: carved from a few large slabs (one cudaMalloc per
// slab instead of one per array; every array starts on a 256-byte boundary)
struct DevAlloc {
    size_t slab = (size_t)1 << 20;   // size of a new slab (at least the request)
    std::vector<void *> ptrs;
    char *cur = nullptr;
    size_t left = 0;
    ~DevAlloc() { release(); }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
        cur = nullptr;
        left = 0;
    }
    template <class T> int get(T *&p, int64_t n)
    {
        const size_t bytes = ((size_t)std::max<int64_t>(n, 1) * sizeof(T) + 255) & ~(size_t)255;
        if (bytes > left) {
            void *q = nullptr;
            size_t sz = std::max(bytes, slab);
            cudaError_t e = cudaMalloc(&q, sz);
            if (e != cudaSuccess && sz > bytes) {
                // no room for a whole slab: this and later arrays get their own
                cudaGetLastError();
                slab = 0;
                sz = bytes;
                e = cudaMalloc(&q, sz);
            }
            if (e != cudaSuccess) {
                p = nullptr;
                return fail(MCGB_E_OOM, std::string("device allocation: ") + cudaGetErrorString(e));
            }
            ptrs.push_back(q);
            cur = (char *)q;
            left = sz;
        }
        p = (T *)cur;
        cur += bytes;
        left -= bytes;
        return MCGB_OK;
    }
};

struct GradGen {          // what the replay needs from one forward generation
    int64_t n = 0, M = 0;
    double *own = nullptr;
    int *nfis = nullptr, *off = nullptr, *perm = nullptr;
    Bank bank{};          // this generation's sites (unsorted) = next generation's births
};

struct EigenRun {            // a power iteration in progress
    bool on = false;
    int64_t N = 0;
    int inactive = 0, active = 0, ncyc = 0, cyc = 0, cur = 0;
    uint64_t seed = 0;
    uint64_t seed_arg = 0;   // as given to mcgb_eigen_begin (checkpoints)
};

struct RunState {
    DevAlloc mem;
    int64_t cap_p = 0, cap_b = 0, cap_acc = 0;
    Particles P{};
    Bank bank[2]{};
    int *list[2] = {nullptr, nullptr};
    int *q_cross = nullptr, *q_coll = nullptr, *off = nullptr, *perm = nullptr, *src_idx = nullptr;
    int *scratch = nullptr, *M = nullptr, *work = nullptr;
    int64_t *gen_base[2] = {nullptr, nullptr};
    double *tacc = nullptr, *tsum = nullptr, *tsum2 = nullptr, *kout = nullptr;
    unsigned long long *cnt = nullptr;
    int *bank_n = nullptr, *err = nullptr, *q_n = nullptr;
    int *pinned = nullptr;   // host-pinned mirror of small counters
};

struct mcgb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mcgb_opts opts{};
    int sms = 1;
    ProblemDef def;
    std::unique_ptr<DeviceWorld> world;
    RunState rs;
    int64_t launches = 0;
    // the device world was built from the definition as it stood at def_version
    int64_t def_version = 0, world_version = -1;
    // device-side material updates: validity flag, checked before the next run
    DevAlloc upd_mem;
    int *upd_bad = nullptr;
    bool upd_pending = false;
    // results
    double k[6] = {0, 0, 0, 0, 0, 0};
    std::vector<double> cyc_ktl, cyc_kc;
    std::vector<int64_t> cyc_m;
    std::vector<std::vector<double>> t_mean, t_sd;
    mcgb_counters counters{};
    std::vector<int32_t> h_coll, h_cross, h_fis, h_fate, h_g;
    std::vector<uint64_t> h_rng;
    std::vector<double> b_xyz;
    std::vector<int64_t> b_parent;
    std::vector<int32_t> b_child, b_mat;
    std::vector<double> cyc_tms, cyc_ms;   // per-cycle device time: transport, whole cycle
    std::vector<cudaEvent_t> events;
    EigenRun eig;
    // persistent cycles replayed as CUDA graphs (two: the banks alternate)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaGraph_t graph_src[2] = {nullptr, nullptr};
    cudaGraphNode_t graph_mark[2] = {nullptr, nullptr};   // event record after the transport
    cudaEvent_t mark_ev[2] = {nullptr, nullptr};
    int graph_launches = 0;                // kernels in one graph
    // event mode: device time of each generation's first flight launch (the
    // whole generation in one k_advance launch over the identity list)
    cudaEvent_t adv_ev[2] = {nullptr, nullptr};
    double adv_ms = 0.0;
    int64_t adv_n = 0, adv_launches = 0;
    cudaStream_t cap_stream = nullptr;
    DevAlloc gmem;                         // cycle counter, draws, bank sizes
    int *cyc_dev = nullptr;
    double *xi_dev = nullptr;
    int64_t *bankm_dev = nullptr;
    int *pinned_cyc = nullptr;
    // derivative forward state
    std::vector<GradGen> grad_gens;
    DevAlloc grad_mem;
    int64_t grad_n = 0;
    int grad_cell = -1;
    bool grad_ready = false;
    // one rank's slice of a sharded power iteration
    struct {
        bool on = false;
        int64_t N = 0, j0 = 0, n = 0, M = 0;
        int inactive = 0, ncyc = 0, cyc = 0;
        int state = 0;               // 0: transport next, 1: export next, 2: import next
        DevAlloc mem;
        double *sums = nullptr;      // the rank's [k_tl, k_c, tally...] sums of the last cycle
    } shard;
    // one rank's slab of a spatially decomposed power iteration
    struct {
        bool on = false;
        int64_t N = 0, cap = 0, M = 0, n_out = 0;
        int inactive = 0, ncyc = 0, cyc = 0, rank = 0, nd = 1;
        int state = 0;               // 0: sources next, 1: sweeping, 2: import next
        DomainCut cut{};
        DevAlloc mem;
        double *cuts = nullptr;
        int *list = nullptr, *n_list = nullptr, *outbox = nullptr, *n_out_dev = nullptr;
        int *work = nullptr;
        ShardSite *glob = nullptr;   // the last cycle's global (parent, child)-ordered bank
    } dom;
};

struct mcgb_batch {
    mcgb_opts opts{};
    int device = 0;
    std::vector<std::unique_ptr<ProblemDef>> defs;
    std::vector<ProblemRun> runs;
    std::unique_ptr<mcgb_ctx> engine;    // owns the device state of batched runs
    std::vector<std::vector<std::vector<double>>> t_mean, t_sd;   // [problem][tally][...]
    mcgb_tune tuned{};
    bool has_tune = false;
};

// ---------------------------------------------------------------------------
static int prepare_buffers(mcgb_ctx *c, int64_t cap_p, int64_t cap_b)
{
    RunState &r = c->rs;
    int acc = c->world->acc_size * c->world->nrep;
    if (cap_p <= r.cap_p && cap_b <= r.cap_b && acc <= r.cap_acc) return MCGB_OK;
    r.mem.release();
    cap_p = std::max(cap_p, r.cap_p);
    cap_b = std::max(cap_b, r.cap_b);
    Particles &P = r.P;
    DevAlloc &m = r.mem;
    // one slab holds every array below (29 per particle, 13 per bank site in
    // each of two banks, lists, queues, scan scratch, tallies)
    m.slab = 8 * (size_t)(40 * cap_p + 28 * cap_b) + 8 * (size_t)std::max(acc, 1) * 3 + ((size_t)16 << 20);
    CKR(m.get(P.x, cap_p)); CKR(m.get(P.y, cap_p)); CKR(m.get(P.z, cap_p));
    CKR(m.get(P.u, cap_p)); CKR(m.get(P.v, cap_p)); CKR(m.get(P.w, cap_p));
    CKR(m.get(P.E, cap_p)); CKR(m.get(P.kt, cap_p)); CKR(m.get(P.kc, cap_p)); CKR(m.get(P.t, cap_p));
    CKR(m.get(P.drem, cap_p));
    CKR(m.get(P.iu, cap_p)); CKR(m.get(P.iv, cap_p)); CKR(m.get(P.iw, cap_p));
    CKR(m.get(P.s, cap_p));
    CKR(m.get(P.g, cap_p)); CKR(m.get(P.cell, cap_p)); CKR(m.get(P.ix, cap_p));
    CKR(m.get(P.iy, cap_p)); CKR(m.get(P.ucell, cap_p)); CKR(m.get(P.mat, cap_p));
    CKR(m.get(P.uk, cap_p)); CKR(m.get(P.prob, cap_p)); CKR(m.get(P.root, cap_p));
    CKR(m.get(P.nfis, cap_p)); CKR(m.get(P.ncoll, cap_p)); CKR(m.get(P.ncross, cap_p));
    CKR(m.get(P.bwhich, cap_p)); CKR(m.get(P.bkind, cap_p)); CKR(m.get(P.fate, cap_p));
    P.cap = cap_p;
    for (int b = 0; b < 2; b++) {
        Bank &B = r.bank[b];
        CKR(m.get(B.x, cap_b)); CKR(m.get(B.y, cap_b)); CKR(m.get(B.z, cap_b)); CKR(m.get(B.t, cap_b));
        CKR(m.get(B.cell, cap_b)); CKR(m.get(B.ix, cap_b)); CKR(m.get(B.iy, cap_b));
        CKR(m.get(B.ucell, cap_b)); CKR(m.get(B.mat, cap_b)); CKR(m.get(B.parent, cap_b));
        CKR(m.get(B.child, cap_b)); CKR(m.get(B.root, cap_b)); CKR(m.get(B.prob, cap_b));
        B.cap = cap_b;
        CKR(m.get(r.list[b], cap_p));
        CKR(m.get(r.gen_base[b], 4096 + 1));
    }
    int64_t big = std::max(cap_p, cap_b);
    CKR(m.get(r.q_cross, cap_p)); CKR(m.get(r.q_coll, cap_p));
    CKR(m.get(r.off, cap_p + 1)); CKR(m.get(r.perm, cap_b)); CKR(m.get(r.src_idx, big));
    CKR(m.get(r.scratch, scan_scratch_ints(cap_p) + 16));
    CKR(m.get(r.M, 4)); CKR(m.get(r.work, 4));
    CKR(m.get(r.tacc, std::max(acc, 1))); CKR(m.get(r.tsum, std::max(c->world->acc_size, 1)));
    CKR(m.get(r.tsum2, std::max(c->world->acc_size, 1)));
    CKR(m.get(r.kout, 2 * 4096)); CKR(m.get(r.cnt, 8));
    CKR(m.get(r.bank_n, 4)); CKR(m.get(r.err, 4)); CKR(m.get(r.q_n, 4));
    if (!r.pinned) CK(cudaMallocHost((void **)&r.pinned, 16 * sizeof(int)));
    r.cap_p = cap_p;
    r.cap_b = cap_b;
    r.cap_acc = acc;
    return MCGB_OK;
}

static RunBufs run_bufs(mcgb_ctx *c, double *own, int own_cell, int own_G)
{
    RunBufs R{};
    R.kacc = nullptr;
    R.tacc = c->rs.tacc;
    R.bank_n = c->rs.bank_n;
    R.err = c->rs.err;
    R.q_n = c->rs.q_n;
    R.own = own;
    R.own_cell = own_cell;
    R.own_G = own_G;
    return R;
}

// Threads per block of the launches over a generation's slots (births, the
// event and segment kernels, the register-resident persistent variant): 128
// by default, which ends the event form's flight launch sooner than 256
// (finer blocks leave less of the last wave idle).
static int block_size(mcgb_ctx *c) { return c->opts.block > 0 ? c->opts.block : 128; }

// The default persistent pool by the physics the world holds (measured on the
// lattice, the continuous-energy pin and the time benchmark): 256 particles per
// 128-thread block for multigroup worlds, 256 per 256-thread block for
// continuous energy, 512 per 256-thread block with time dependence as well.
static int default_pool(const World &W)
{
    if (!W.ce_any) return 2256;
    return W.time_any ? 512 : 256;
}

// Transport one cycle / generation of `total` slots (host-known bound).
static int transport_generation(mcgb_ctx *c, const RunBufs &R, int gen, int64_t total,
                                const int64_t *gen_base, const int *src_idx, int eigen,
                                const Bank &Bsrc, const Bank &Bdst, cudaStream_t st = nullptr,
                                const int *gen_dev = nullptr)
{
    RunState &r = c->rs;
    const World &W = c->world->W;
    if (!st) st = c->stream;
    int block = block_size(c);
    if (c->opts.mode == MCGB_MODE_PERSISTENT) {
        CK(cudaMemsetAsync(r.work, 0, sizeof(int), st));
        PersistentArgs a{};
        a.total = total;
        a.gen_n = nullptr;
        a.work = r.work;
        a.max_passes = c->opts.max_iterations > 0 ? c->opts.max_iterations : 0;
        // every slot's birth made at once by a grid over the generation, so that
        // a block's refill copies a ready state instead of waiting on the bank
        // reads, the stream skip-ahead and the sampling of each birth
        launch_source(W, r.P, Bsrc, R, gen, total, gen_base, src_idx, eigen, block, st, gen_dev);
        c->launches += 1;
        int pool = c->opts.pool == 0 ? default_pool(W) : c->opts.pool;
        if (pool > 0) {
            int bps = c->opts.blocks_per_sm > 0 ? c->opts.blocks_per_sm
                                                 : std::max(1, pool_max_blocks_per_sm(pool, W.ce_any != 0));
            int ppb = pool_particles_per_block(pool);
            int64_t want = (total + ppb - 1) / ppb;
            int grid = (int)std::min<int64_t>((int64_t)c->sms * bps, std::max<int64_t>(want, 1));
            if (!launch_pool(W, r.P, Bsrc, Bdst, R, a, pool, grid, st))
                return fail(MCGB_E_INVALID_ARG, "unknown pool variant");
        } else {
            int bps = c->opts.blocks_per_sm > 0 ? c->opts.blocks_per_sm
                                                 : std::max(1, persistent_max_blocks_per_sm(block));
            int64_t want = (total + block - 1) / block;
            int grid = (int)std::min<int64_t>((int64_t)c->sms * bps, std::max<int64_t>(want, 1));
            launch_persistent(W, r.P, Bsrc, Bdst, R, a, grid, block, st);
        }
        c->launches += 1;
        CK(cudaGetLastError());
        return MCGB_OK;
    }
    launch_source(W, r.P, Bsrc, R, gen, total, gen_base, src_idx, eigen, block, st);
    c->launches += 1;
    // Host-driven iterations over compacted lists.  The length of list b is kept
    // on the device in q_n[2 + b]; kernels read it there and their grids cover
    // the last length the host has seen (lists only shrink within a generation),
    // so the host reads the length back only every SYNC_EVERY iterations.
    const int SYNC_EVERY = 16;
    if (c->opts.mode == MCGB_MODE_EVENT && !c->adv_ev[0]) {
        CK(cudaEventCreate(&c->adv_ev[0]));
        CK(cudaEventCreate(&c->adv_ev[1]));
    }
    int64_t bound = total;
    int cur = 0;
    const int *list = nullptr;   // identity for the first iteration
    const int *n_dev = nullptr;
    int64_t maxit = c->opts.max_iterations > 0 ? c->opts.max_iterations : 10000000;
    for (int64_t it = 0;; it++) {
        if (it >= maxit) {
            // the queued launches finish on their own (each is bounded); the
            // stream is drained so that the caller may reuse the context
            CK(cudaStreamSynchronize(st));
            return fail(MCGB_E_TIMEOUT, "event iteration limit reached");
        }
        int *next = r.list[cur];
        int *next_n = r.q_n + 2 + cur;
        CK(cudaMemsetAsync(r.q_n, 0, 2 * sizeof(int), st));
        CK(cudaMemsetAsync(next_n, 0, sizeof(int), st));
        if (c->opts.mode == MCGB_MODE_SEGMENT) {
            launch_segment(W, r.P, Bdst, R, list, (int)bound, n_dev, next, next_n, block, st);
            c->launches += 1;
        } else {
            const bool timed = it == 0 && c->adv_ev[0];
            if (timed) CK(cudaEventRecord(c->adv_ev[0], st));
            launch_advance(W, r.P, R, list, (int)bound, n_dev, r.q_cross, r.q_coll, block, st);
            if (timed) CK(cudaEventRecord(c->adv_ev[1], st));
            launch_cross(W, r.P, R, r.q_cross, (int)bound, next, next_n, block, st);
            launch_collide(W, r.P, Bdst, R, r.q_coll, (int)bound, next, next_n, block, st);
            c->launches += 3;
        }
        c->counters.event_iterations++;
        list = next;
        n_dev = next_n;
        cur ^= 1;
        if (it % SYNC_EVERY == SYNC_EVERY - 1 || it == 0) {
            CK(cudaMemcpyAsync(r.pinned, next_n, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (it == 0 && c->opts.mode == MCGB_MODE_EVENT && c->adv_ev[0]) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, c->adv_ev[0], c->adv_ev[1]));
                c->adv_ms += ms;
                c->adv_n += total;
                c->adv_launches += 1;
            }
            bound = r.pinned[0];
            if (bound == 0) break;
        }
    }
    CK(cudaGetLastError());
    return MCGB_OK;
}

static void mean_sd(double sum, double sum2, int n, double &mean, double &sd)
{
    mean = sum / n;
    if (n > 1) {
        double var = (sum2 - n * mean * mean) / (n - 1);
        sd = std::sqrt(var > 0.0 ? var / n : 0.0);
    } else {
        sd = 0.0;
    }
}

static double draw_host(uint64_t &s)
{
    s = rng_next(s);
    return (double)((s >> 10) + 1) * 0x1p-53;
}

static int fetch_counters(mcgb_ctx *c)
{
    unsigned long long h[8];
    CK(cudaMemcpyAsync(h, c->rs.cnt, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->counters.collisions = (int64_t)h[0];
    c->counters.crossings = (int64_t)h[1];
    c->counters.leaks = (int64_t)h[2];
    c->counters.lost = (int64_t)h[3];
    c->counters.capped = (int64_t)h[4];
    c->counters.time_cut = (int64_t)h[5];
    c->counters.kernel_launches = c->launches;
    c->counters.world_bytes = c->world ? (int64_t)c->world->bytes : 0;
    return MCGB_OK;
}

static int copy_records(mcgb_ctx *c, int64_t n)
{
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    c->h_coll.resize(n); c->h_cross.resize(n); c->h_fis.resize(n);
    c->h_fate.resize(n); c->h_g.resize(n); c->h_rng.resize(n);
    std::vector<signed char> fate(n);
    CK(cudaMemcpyAsync(c->h_coll.data(), r.P.ncoll, n * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->h_cross.data(), r.P.ncross, n * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->h_fis.data(), r.P.nfis, n * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->h_g.data(), r.P.g, n * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->h_rng.data(), r.P.s, n * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(fate.data(), r.P.fate, n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int64_t j = 0; j < n; j++) c->h_fate[j] = fate[j];
    return MCGB_OK;
}

// the bank `B` of M sites with permutation perm, copied in (parent, child) order
static int copy_bank(mcgb_ctx *c, const Bank &B, int64_t M)
{
    cudaStream_t st = c->stream;
    std::vector<int> perm(M), par(M), ch(M), mat(M);
    std::vector<double> x(M), y(M), z(M);
    if (M > 0) {
        CK(cudaMemcpyAsync(perm.data(), c->rs.perm, M * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(par.data(), B.parent, M * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ch.data(), B.child, M * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(mat.data(), B.mat, M * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(x.data(), B.x, M * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(y.data(), B.y, M * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(z.data(), B.z, M * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    c->b_xyz.resize(3 * M); c->b_parent.resize(M); c->b_child.resize(M); c->b_mat.resize(M);
    for (int64_t k = 0; k < M; k++) {
        int b = perm[k];
        c->b_xyz[3 * k] = x[b]; c->b_xyz[3 * k + 1] = y[b]; c->b_xyz[3 * k + 2] = z[b];
        c->b_parent[k] = par[b]; c->b_child[k] = ch[b]; c->b_mat[k] = mat[b];
    }
    return MCGB_OK;
}

static int read_flags(mcgb_ctx *c, int64_t &M, int &err)
{
    CK(cudaMemcpyAsync(c->rs.pinned + 4, c->rs.M, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->rs.pinned + 5, c->rs.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->rs.pinned + 6, c->rs.bank_n, sizeof(int), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    M = c->rs.pinned[4];
    err = c->rs.pinned[5];
    if (c->rs.pinned[6] > c->rs.cap_b) err |= ERR_BANK_OVERFLOW;
    return MCGB_OK;
}

static int build_single(mcgb_ctx *c, int64_t n, int batches, uint64_t seed)
{
    if (!c->world) c->world.reset(new DeviceWorld());
    c->world_version = -1;
    c->upd_pending = false;   // a rebuilt world holds the host definition's tables
    std::vector<ProblemRun> runs{{&c->def, n, batches, seed}};
    std::string e = build_world(runs, *c->world, c->stream);
    if (!e.empty()) return fail(MCGB_E_STATE, e);
    c->world_version = c->def_version;
    return MCGB_OK;
}

static int check_lost(mcgb_ctx *c)
{
    if (c->counters.lost > 0 && (double)c->counters.lost > 1e-6 * (double)c->counters.histories)
        return fail(MCGB_E_LOST_PARTICLES, "lost particles: " + std::to_string(c->counters.lost));
    return MCGB_OK;
}

// ---------------------------------------------------------------------------
// k-eigenvalue power iteration, stepwise: begin, any number of cycles, finish.
static void drop_cycle_graphs(mcgb_ctx *c)
{
    for (int q = 0; q < 2; q++)
        if (c->graph[q]) {
            cudaGraphExecDestroy(c->graph[q]);
            c->graph[q] = nullptr;
        }
}

static int eigen_begin(mcgb_ctx *c, int64_t N, int inactive, int active, uint64_t seed)
{
    if (N <= 0 || N > (int64_t)1 << 30 || active < 1 || inactive < 0 || inactive + active > 4096)
        return fail(MCGB_E_INVALID_ARG, "bad run size");
    if (c->def.time_on) return fail(MCGB_E_INVALID_ARG, "time dependence is for fixed-source runs");
    c->eig.on = false;
    CKR(build_single(c, N, 1, seed));
    double bf = c->opts.bank_factor > 0 ? c->opts.bank_factor : 3.0;
    int64_t cap_b = (int64_t)(bf * (double)N) + 1024;
    CKR(prepare_buffers(c, N, cap_b));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    int acc = W.acc_size;
    CK(cudaMemsetAsync(r.tacc, 0, sizeof(double) * (size_t)acc * W.nrep, st));
    CK(cudaMemsetAsync(r.tsum, 0, sizeof(double) * std::max(acc, 1), st));
    CK(cudaMemsetAsync(r.tsum2, 0, sizeof(double) * std::max(acc, 1), st));
    CK(cudaMemsetAsync(r.kout, 0, sizeof(double) * 2 * 4096, st));
    CK(cudaMemsetAsync(r.cnt, 0, sizeof(unsigned long long) * 8, st));
    CK(cudaMemsetAsync(r.err, 0, sizeof(int), st));
    int64_t base[2] = {0, N};
    CK(cudaMemcpyAsync(r.gen_base[0], base, sizeof base, cudaMemcpyHostToDevice, st));
    int ncyc = inactive + active;
    c->counters = mcgb_counters{};
    c->counters.world_bytes = (int64_t)c->world->bytes;
    c->launches = 0;
    c->cyc_ktl.assign(ncyc, 0.0);
    c->cyc_kc.assign(ncyc, 0.0);
    c->cyc_m.assign(ncyc, 0);
    c->cyc_tms.assign(ncyc, 0.0);
    c->cyc_ms.assign(ncyc, 0.0);
    EigenRun &e = c->eig;
    e.on = true;
    e.N = N;
    e.inactive = inactive;
    e.active = active;
    e.ncyc = ncyc;
    e.cyc = 0;
    e.cur = 0;
    e.seed = c->world->probs[0].seed;
    e.seed_arg = seed;
    // device copies for graph replay: the resampling draw of every cycle, bank sizes
    drop_cycle_graphs(c);
    c->gmem.release();
    CKR(c->gmem.get(c->cyc_dev, 1));
    CKR(c->gmem.get(c->xi_dev, ncyc));
    CKR(c->gmem.get(c->bankm_dev, ncyc));
    {
        std::vector<double> xi(ncyc);
        for (int q = 0; q < ncyc; q++) {
            uint64_t rs = rng_stream(e.seed, ((uint64_t)q << 32) + 0xFFFFFFFFULL);
            xi[q] = draw_host(rs);
        }
        CK(cudaMemcpyAsync(c->xi_dev, xi.data(), sizeof(double) * ncyc, cudaMemcpyHostToDevice, st));
        if (c->pinned_cyc) cudaFreeHost(c->pinned_cyc);
        CK(cudaMallocHost((void **)&c->pinned_cyc, sizeof(int) * ncyc));
        for (int q = 0; q < ncyc; q++) c->pinned_cyc[q] = q;
        CK(cudaStreamSynchronize(st));
    }
    if (c->events.size() < (size_t)3 * ncyc + 3) {
        size_t old = c->events.size();
        c->events.resize(3 * ncyc + 3);
        for (size_t i = old; i < c->events.size(); i++) CK(cudaEventCreate(&c->events[i]));
    }
    return MCGB_OK;
}

// Capture one cycle (source from the bank, transport, bank order, resampling,
// statistics) as a graph per bank parity; the cycle index, its resampling
// draw and the active flag are read on the device, and the graph's last
// kernel records the bank size and advances the cycle index.
static int capture_cycle_graphs(mcgb_ctx *c);

// Both cycle graphs, or neither: a failed capture or instantiation leaves no
// graph behind, so the next call captures again from the start.
static int build_cycle_graphs(mcgb_ctx *c)
{
    int rc = capture_cycle_graphs(c);
    if (rc != MCGB_OK) drop_cycle_graphs(c);
    return rc;
}

static int capture_cycle_graphs(mcgb_ctx *c)
{
    EigenRun &e = c->eig;
    RunState &r = c->rs;
    const World &W = c->world->W;
    RunBufs R = run_bufs(c, nullptr, -1, 0);
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = c->cap_stream;
    for (int parity = 0; parity < 2; parity++) {
        int64_t l0 = c->launches;
        if (!c->mark_ev[parity]) CK(cudaEventCreate(&c->mark_ev[parity]));
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        cudaMemsetAsync(r.bank_n, 0, sizeof(int), cs);
        int rc = transport_generation(c, R, 0, e.N, r.gen_base[0], r.src_idx, 1, r.bank[parity],
                                      r.bank[parity ^ 1], cs, c->cyc_dev);
        cudaEventRecordWithFlags(c->mark_ev[parity], cs, cudaEventRecordExternal);
        launch_reduce_gen(r.P, e.N, nullptr, r.kout, r.cnt, cs, c->cyc_dev);
        scan_exclusive(r.P.nfis, r.off, e.N, r.M, r.scratch, cs);
        launch_perm(r.bank[parity ^ 1], r.off, r.M, r.perm, c->sms * 4, cs);
        launch_resample_dev(r.perm, r.M, e.N, c->xi_dev, c->cyc_dev, r.src_idx, r.err,
                            r.bank[parity ^ 1].cap, cs);
        launch_tally_cycle(r.tacc, W.acc_size, W.nrep, (double)e.N, 0, r.tsum, r.tsum2, cs,
                           c->cyc_dev, e.inactive);
        launch_cycle_end(c->cyc_dev, r.M, c->bankm_dev, cs);
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(cs, &g);
        if (rc != MCGB_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CK(ee);
        // the event-record node after the transport kernel, re-pointed per cycle
        size_t nn = 0;
        CK(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(g, nodes.data(), &nn));
        c->graph_mark[parity] = nullptr;
        for (cudaGraphNode_t n : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(n, &ty));
            if (ty == cudaGraphNodeTypeEventRecord) c->graph_mark[parity] = n;
        }
        ee = cudaGraphInstantiate(&c->graph[parity], g, 0);
        if (c->graph_src[parity]) cudaGraphDestroy(c->graph_src[parity]);
        c->graph_src[parity] = g;
        CK(ee);
        int ntiles = (int)((e.N + 4095) / 4096);
        c->graph_launches = (int)(c->launches - l0) + 1 + (ntiles > 1 ? 3 : 2) + 3 +
                            (W.acc_size > 0 ? 1 : 0);
        c->launches = l0;
    }
    return MCGB_OK;
}

static bool use_graphs(const mcgb_ctx *c)
{
    return c->opts.mode == MCGB_MODE_PERSISTENT && c->opts.graphs >= 0;
}

static int eigen_cycles(mcgb_ctx *c, int k)
{
    EigenRun &e = c->eig;
    if (!e.on) return fail(MCGB_E_STATE, "no eigenvalue run in progress");
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    RunBufs R = run_bufs(c, nullptr, -1, 0);
    int64_t N = e.N;
    // cycles after the first: graph launches back to back, checked once at the end
    if (use_graphs(c) && e.cyc >= 1 && k > 0 && e.cyc < e.ncyc) {
        if (!c->graph[0] || !c->graph[1]) CKR(build_cycle_graphs(c));
        int first = e.cyc;
        CK(cudaMemcpyAsync(c->cyc_dev, c->pinned_cyc + first, sizeof(int), cudaMemcpyHostToDevice, st));
        int last = std::min(e.ncyc, first + k);
        for (int cyc = first; cyc < last; cyc++) {
            int par = cyc & 1;
            if (c->graph_mark[par])
                CK(cudaGraphExecEventRecordNodeSetEvent(c->graph[par], c->graph_mark[par],
                                                        c->events[3 * cyc + 1]));
            CK(cudaEventRecord(c->events[3 * cyc], st));
            CK(cudaGraphLaunch(c->graph[par], st));
            CK(cudaEventRecord(c->events[3 * cyc + 2], st));
            c->launches += c->graph_launches;
        }
        std::vector<int64_t> bm(last - first);
        CK(cudaMemcpyAsync(bm.data(), c->bankm_dev + first, sizeof(int64_t) * (last - first),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(r.pinned + 5, r.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        int err = r.pinned[5];
        for (int cyc = first; cyc < last; cyc++) {
            float t1 = 0.f, t2 = 0.f;
            if (c->graph_mark[cyc & 1]) cudaEventElapsedTime(&t1, c->events[3 * cyc], c->events[3 * cyc + 1]);
            cudaEventElapsedTime(&t2, c->events[3 * cyc], c->events[3 * cyc + 2]);
            c->cyc_ms[cyc] = t2;
            c->cyc_tms[cyc] = t1;
            c->cyc_m[cyc] = bm[cyc - first];
        }
        e.cyc = last;
        if (err & ERR_BANK_OVERFLOW) {
            e.on = false;
            return fail(MCGB_E_BANK_OVERFLOW, "fission bank overflow");
        }
        if (err & ERR_SOURCE) {
            e.on = false;
            return fail(MCGB_E_STATE, "source sampling failed");
        }
        if (err & ERR_ITER) {
            e.on = false;
            return fail(MCGB_E_TIMEOUT, "persistent event loop pass limit reached");
        }
        for (int cyc = first; cyc < last; cyc++)
            if (c->cyc_m[cyc] == 0) {
                e.on = false;
                return fail(MCGB_E_STATE, "fission bank empty after cycle " + std::to_string(cyc));
            }
        e.cur = last & 1;
        if (last == e.ncyc && c->opts.record_histories) {
            CKR(copy_records(c, N));
            CKR(copy_bank(c, r.bank[e.cur], c->cyc_m[last - 1]));
        }
        return MCGB_OK;
    }
    for (int q = 0; q < k && e.cyc < e.ncyc; q++) {
        int cyc = e.cyc;
        int nxt = e.cur ^ 1;
        cudaEvent_t ev0 = c->events[3 * cyc], ev1 = c->events[3 * cyc + 1], ev2 = c->events[3 * cyc + 2];
        CK(cudaEventRecord(ev0, st));
        CK(cudaMemsetAsync(r.bank_n, 0, sizeof(int), st));
        CKR(transport_generation(c, R, cyc, N, r.gen_base[0], cyc == 0 ? nullptr : r.src_idx, 1,
                                 r.bank[e.cur], r.bank[nxt]));
        CK(cudaEventRecord(ev1, st));
        launch_reduce_gen(r.P, N, nullptr, r.kout + 2 * cyc, r.cnt, st);
        scan_exclusive(r.P.nfis, r.off, N, r.M, r.scratch, st);
        launch_perm(r.bank[nxt], r.off, r.M, r.perm, c->sms * 4, st);
        uint64_t rs = rng_stream(e.seed, ((uint64_t)cyc << 32) + 0xFFFFFFFFULL);
        double xi = draw_host(rs);
        launch_resample(r.perm, r.M, N, xi, r.src_idx, r.err, r.bank[nxt].cap, st);
        launch_tally_cycle(r.tacc, W.acc_size, W.nrep, (double)N, cyc >= e.inactive, r.tsum, r.tsum2, st);
        c->launches += 7;
        CK(cudaEventRecord(ev2, st));
        CK(cudaGetLastError());
        // the later cycles' graphs are captured while the first cycle runs; a
        // failed capture is reported once this cycle's results are recorded
        int graph_rc = MCGB_OK;
        if (cyc == 0 && use_graphs(c) && !c->graph[0] && e.ncyc > 1) graph_rc = build_cycle_graphs(c);
        int64_t M;
        int err;
        CKR(read_flags(c, M, err));
        c->cyc_m[cyc] = M;
        float t1 = 0.f, t2 = 0.f;
        cudaEventElapsedTime(&t1, ev0, ev1);
        cudaEventElapsedTime(&t2, ev0, ev2);
        c->cyc_tms[cyc] = t1;
        c->cyc_ms[cyc] = t2;
        e.cyc++;
        if (err & ERR_BANK_OVERFLOW) {
            e.on = false;
            return fail(MCGB_E_BANK_OVERFLOW, "fission bank overflow in cycle " + std::to_string(cyc));
        }
        if (err & ERR_SOURCE) {
            e.on = false;
            return fail(MCGB_E_STATE, "source sampling failed");
        }
        if (err & ERR_ITER) {
            e.on = false;
            return fail(MCGB_E_TIMEOUT, "persistent event loop pass limit reached in cycle " +
                                            std::to_string(cyc));
        }
        if (cyc == e.ncyc - 1 && c->opts.record_histories) {
            CKR(copy_records(c, N));
            CKR(copy_bank(c, r.bank[nxt], M));
        }
        if (M == 0) {
            e.on = false;
            return fail(MCGB_E_STATE, "fission bank empty after cycle " + std::to_string(cyc));
        }
        e.cur = nxt;
        if (graph_rc != MCGB_OK) return graph_rc;
    }
    return MCGB_OK;
}

static int eigen_finish(mcgb_ctx *c)
{
    EigenRun &e = c->eig;
    if (!e.on) return fail(MCGB_E_STATE, "no eigenvalue run in progress");
    if (e.cyc < e.ncyc) return fail(MCGB_E_STATE, "cycles remain to be run");
    e.on = false;
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    int acc = c->world->W.acc_size;
    int ncyc = e.ncyc, inactive = e.inactive, active = e.active;
    int64_t N = e.N;
    std::vector<double> kout(2 * ncyc);
    CK(cudaMemcpyAsync(kout.data(), r.kout, sizeof(double) * 2 * ncyc, cudaMemcpyDeviceToHost, st));
    std::vector<double> ts(std::max(acc, 1)), ts2(std::max(acc, 1));
    CK(cudaMemcpyAsync(ts.data(), r.tsum, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ts2.data(), r.tsum2, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double ks[3] = {0, 0, 0}, ks2[3] = {0, 0, 0};
    for (int cyc = 0; cyc < ncyc; cyc++) {
        c->cyc_ktl[cyc] = kout[2 * cyc] / (double)N;
        c->cyc_kc[cyc] = kout[2 * cyc + 1] / (double)N;
        if (cyc >= inactive) {
            double kv[3] = {c->cyc_ktl[cyc], c->cyc_kc[cyc], (double)c->cyc_m[cyc] / (double)N};
            for (int q = 0; q < 3; q++) {
                ks[q] += kv[q];
                ks2[q] += kv[q] * kv[q];
            }
        }
    }
    for (int q = 0; q < 3; q++) mean_sd(ks[q], ks2[q], active, c->k[2 * q], c->k[2 * q + 1]);
    DeviceWorld &dw = *c->world;
    c->t_mean.assign(c->def.tallies.size(), {});
    c->t_sd.assign(c->def.tallies.size(), {});
    for (size_t t = 0; t < c->def.tallies.size(); t++) {
        int gt = dw.tally_first[0] + (int)t;
        int nb = dw.t_nbins[gt] * dw.t_ne[gt] * std::max(1, dw.t_ntb[gt]);
        c->t_mean[t].resize(nb);
        c->t_sd[t].resize(nb);
        for (int b = 0; b < nb; b++)
            mean_sd(ts[dw.t_off[gt] + b], ts2[dw.t_off[gt] + b], active, c->t_mean[t][b],
                    c->t_sd[t][b]);
    }
    c->counters.histories = N * ncyc;
    c->counters.generations = ncyc;
    CKR(fetch_counters(c));
    return check_lost(c);
}

static int run_eigen(mcgb_ctx *c, int64_t N, int inactive, int active, uint64_t seed)
{
    CKR(eigen_begin(c, N, inactive, active, seed));
    CKR(eigen_cycles(c, inactive + active));
    return eigen_finish(c);
}

// Fixed source over the problems of the current world (one or a batch).
// With `grad`, keeps every generation's own detector tallies and banks.
static int run_fixed_world(mcgb_ctx *c, bool grad, int det_cell)
{
    DeviceWorld &dw = *c->world;
    const World &W = dw.W;
    int nprob = W.nprob;
    int64_t N = 0;
    std::vector<int64_t> base(nprob + 1, 0);
    for (int p = 0; p < nprob; p++) base[p + 1] = base[p] + dw.probs[p].n;
    N = base[nprob];
    if (N <= 0 || N > (int64_t)1 << 30) return fail(MCGB_E_INVALID_ARG, "bad run size");
    double bf = c->opts.bank_factor > 0 ? c->opts.bank_factor : 3.0;
    int64_t cap_b = (int64_t)(bf * (double)N) + 1024;
    CKR(prepare_buffers(c, std::max(N, cap_b), cap_b));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    int acc = W.acc_size;
    CK(cudaMemsetAsync(r.tacc, 0, sizeof(double) * (size_t)acc * W.nrep, st));
    CK(cudaMemsetAsync(r.kout, 0, sizeof(double) * 2 * 4096, st));
    CK(cudaMemsetAsync(r.cnt, 0, sizeof(unsigned long long) * 8, st));
    CK(cudaMemsetAsync(r.err, 0, sizeof(int), st));
    CK(cudaMemcpyAsync(r.gen_base[0], base.data(), sizeof(int64_t) * (nprob + 1),
                       cudaMemcpyHostToDevice, st));
    c->counters = mcgb_counters{};
    c->counters.world_bytes = (int64_t)dw.bytes;
    c->launches = 0;
    if (grad) {
        c->grad_gens.clear();
        c->grad_mem.release();
        c->grad_ready = false;
    }
    int G = dw.probs[0].G;
    int cur = 0, gb = 0;
    int64_t total = N;
    const int *src = nullptr;
    int gen;
    const int MAX_GEN = 200;
    for (gen = 0; gen < MAX_GEN; gen++) {
        int nxt = cur ^ 1;
        double *own = nullptr;
        if (grad) {
            CKR(c->grad_mem.get(own, total * G));
            CK(cudaMemsetAsync(own, 0, sizeof(double) * total * G, st));
        }
        RunBufs R = run_bufs(c, own, det_cell, G);
        CK(cudaMemsetAsync(r.bank_n, 0, sizeof(int), st));
        CKR(transport_generation(c, R, gen, total, r.gen_base[gb], src, 0, r.bank[cur], r.bank[nxt]));
        launch_reduce_gen(r.P, total, nullptr, r.kout, r.cnt, st);
        scan_exclusive(r.P.nfis, r.off, total, r.M, r.scratch, st);
        launch_perm(r.bank[nxt], r.off, r.M, r.perm, c->sms * 4, st);
        launch_gen_base(r.gen_base[gb], nprob, r.off, r.M, r.gen_base[gb ^ 1], st);
        c->launches += 6;
        CK(cudaGetLastError());
        int64_t M;
        int err;
        CKR(read_flags(c, M, err));
        c->counters.histories += total;
        if (err & ERR_BANK_OVERFLOW)
            return fail(MCGB_E_BANK_OVERFLOW, "fission bank overflow in generation " + std::to_string(gen) + " (raise opts.bank_factor)");
        if (err & ERR_SOURCE) return fail(MCGB_E_STATE, "source sampling failed");
        if (err & ERR_ITER)
            return fail(MCGB_E_TIMEOUT, "persistent event loop pass limit reached in generation " +
                                            std::to_string(gen));
        if (gen == 0 && c->opts.record_histories) {
            CKR(copy_records(c, total));
            CKR(copy_bank(c, r.bank[nxt], M));
        }
        if (grad) {
            GradGen g;
            g.n = total;
            g.M = M;
            g.own = own;
            CKR(c->grad_mem.get(g.nfis, total));
            CKR(c->grad_mem.get(g.off, total));
            CKR(c->grad_mem.get(g.perm, M));
            CK(cudaMemcpyAsync(g.nfis, r.P.nfis, 4 * total, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(g.off, r.off, 4 * total, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(g.perm, r.perm, 4 * std::max<int64_t>(M, 1), cudaMemcpyDeviceToDevice, st));
            Bank &B = g.bank;
            const Bank &S = r.bank[nxt];
            CKR(c->grad_mem.get(B.x, M)); CKR(c->grad_mem.get(B.y, M)); CKR(c->grad_mem.get(B.z, M));
            CKR(c->grad_mem.get(B.t, M));
            CKR(c->grad_mem.get(B.cell, M)); CKR(c->grad_mem.get(B.ix, M));
            CKR(c->grad_mem.get(B.iy, M)); CKR(c->grad_mem.get(B.ucell, M));
            CKR(c->grad_mem.get(B.mat, M)); CKR(c->grad_mem.get(B.root, M));
            if (M > 0) {
                CK(cudaMemcpyAsync(B.x, S.x, 8 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.y, S.y, 8 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.z, S.z, 8 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.t, S.t, 8 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.cell, S.cell, 4 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.ix, S.ix, 4 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.iy, S.iy, 4 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.ucell, S.ucell, 4 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.mat, S.mat, 4 * M, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(B.root, S.root, 4 * M, cudaMemcpyDeviceToDevice, st));
            }
            B.cap = M;
            c->grad_gens.push_back(g);
        }
        if (M == 0) break;
        // next generation: every site, in (parent, child) order
        CK(cudaMemcpyAsync(r.src_idx, r.perm, 4 * M, cudaMemcpyDeviceToDevice, st));
        src = r.src_idx;
        total = M;
        cur = nxt;
        gb ^= 1;
    }
    if (gen == MAX_GEN) return fail(MCGB_E_TIMEOUT, "generation limit reached");
    c->counters.generations = gen + 1;
    // batch statistics
    std::vector<double> sums(std::max(acc, 1));
    if (acc > 0) {
        launch_acc_reduce(r.tacc, acc, W.nrep, r.tsum, st);
        c->launches += 1;
        CK(cudaMemcpyAsync(sums.data(), r.tsum, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    CKR(fetch_counters(c));
    c->t_mean.clear();
    c->t_sd.clear();
    for (int p = 0; p < nprob; p++) {
        const ProblemDev &P = dw.probs[p];
        int B = P.batches;
        std::vector<int64_t> nb(B, 0);
        for (int64_t j = 0; j < P.n; j++) nb[(j * B) / P.n]++;
        for (int t = 0; t < P.tally_count; t++) {
            int gt = P.tally_first + t;
            int ns = dw.t_nbins[gt] * dw.t_ne[gt] * std::max(1, dw.t_ntb[gt]);
            std::vector<double> mean(ns), sd(ns);
            for (int b = 0; b < ns; b++) {
                double s = 0.0, s2 = 0.0;
                for (int q = 0; q < B; q++) {
                    double v = sums[dw.t_off[gt] + (size_t)q * ns + b];
                    v /= (double)nb[q];
                    s += v;
                    s2 += v * v;
                }
                mean_sd(s, s2, B, mean[b], sd[b]);
            }
            c->t_mean.push_back(mean);
            c->t_sd.push_back(sd);
        }
    }
    if (grad) {
        c->grad_n = N;
        c->grad_cell = det_cell;
        c->grad_ready = true;
    }
    return check_lost(c);
}

// ---------------------------------------------------------------------------
// C ABI
extern "C" {

const char *mcgb_last_error(void) { return g_err.c_str(); }

int mcgb_create(mcgb_ctx **out, const mcgb_opts *opts)
{
    if (!out) return fail(MCGB_E_INVALID_ARG, "null output");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(MCGB_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    std::unique_ptr<mcgb_ctx> c(new mcgb_ctx());
    if (opts) c->opts = *opts;
    if (c->opts.device < 0 || c->opts.device >= ndev) return fail(MCGB_E_INVALID_ARG, "bad device");
    c->device = c->opts.device;
    CK(cudaSetDevice(c->device));
    CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
    if (c->opts.mode < MCGB_MODE_EVENT || c->opts.mode > MCGB_MODE_SEGMENT)
        return fail(MCGB_E_INVALID_ARG, "mode must be MCGB_MODE_EVENT, _PERSISTENT or _SEGMENT");
    if (c->opts.block != 0 && (c->opts.block < 32 || c->opts.block > 256 || c->opts.block % 32))
        return fail(MCGB_E_INVALID_ARG, "block must be a multiple of 32 in [32, 256]");
    {
        int pl = c->opts.pool;
        if (!(pl == 0 || pl == -1 || pl == 32 || pl == 64 || pl == 128 || pl == 256 || pl == 512 ||
              pl == 1024 || pl == 2256 || pl == 2512))
            return fail(MCGB_E_INVALID_ARG,
                        "pool must be 32, 64, 128, 256, 512, 1024, 2256, 2512, 0 or -1");
    }
    *out = c.release();
    return MCGB_OK;
}

int mcgb_destroy(mcgb_ctx *ctx)
{
    if (!ctx) return MCGB_OK;
    cudaSetDevice(ctx->device);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    for (int q = 0; q < 2; q++)
        if (ctx->adv_ev[q]) cudaEventDestroy(ctx->adv_ev[q]);
    for (int q = 0; q < 2; q++) {
        if (ctx->graph[q]) cudaGraphExecDestroy(ctx->graph[q]);
        if (ctx->graph_src[q]) cudaGraphDestroy(ctx->graph_src[q]);
        if (ctx->mark_ev[q]) cudaEventDestroy(ctx->mark_ev[q]);
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->pinned_cyc) cudaFreeHost(ctx->pinned_cyc);
    if (ctx->rs.pinned) cudaFreeHost(ctx->rs.pinned);
    delete ctx;
    return MCGB_OK;
}

int mcgb_set_stream(mcgb_ctx *ctx, void *stream)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    ctx->stream = (cudaStream_t)stream;
    return MCGB_OK;
}

int mcgb_set_mode(mcgb_ctx *ctx, int mode)
{
    if (!ctx || mode < MCGB_MODE_EVENT || mode > MCGB_MODE_SEGMENT)
        return fail(MCGB_E_INVALID_ARG, "bad mode");
    ctx->opts.mode = mode;
    return MCGB_OK;
}

int mcgb_add_surface(mcgb_ctx *ctx, int type, const double coef[4], int bc, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || !coef || type < 0 || type > 5 || bc < 0 || bc > 2)
        return fail(MCGB_E_INVALID_ARG, "bad surface type or boundary");
    if (bc == MCGB_BC_REFLECT && type > MCGB_SURF_PLANE)
        return fail(MCGB_E_INVALID_ARG, "reflective boundaries must be planes");
    if ((type == MCGB_SURF_CYLZ && !(coef[2] > 0.0)) || (type == MCGB_SURF_SPHERE && !(coef[3] > 0.0)))
        return fail(MCGB_E_INVALID_ARG, "radius must be positive");
    ProblemDef &d = ctx->def;
    d.s_type.push_back(type);
    d.s_bc.push_back(bc);
    for (int k = 0; k < 4; k++) d.s_coef.push_back(coef[k]);
    if (id) *id = (int)d.s_type.size() - 1;
    return MCGB_OK;
}

int mcgb_add_cell(mcgb_ctx *ctx, int universe, int n, const int *surf, const int *sense,
                  int fill_kind, int fill, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || universe < 0 || n < 0 || (n > 0 && (!surf || !sense)) || fill < 0 ||
        (fill_kind != MCGB_FILL_MATERIAL && fill_kind != MCGB_FILL_LATTICE))
        return fail(MCGB_E_INVALID_ARG, "bad cell");
    CellDef c;
    c.univ = universe;
    c.fillk = fill_kind;
    c.fill = fill;
    for (int k = 0; k < n; k++) {
        if (surf[k] < 0 || surf[k] >= (int)ctx->def.s_type.size() || (sense[k] != 1 && sense[k] != -1))
            return fail(MCGB_E_INVALID_ARG, "bad half-space");
        c.surf.push_back(surf[k]);
        c.sense.push_back(sense[k]);
    }
    ctx->def.cells.push_back(c);
    if (id) *id = (int)ctx->def.cells.size() - 1;
    return MCGB_OK;
}

int mcgb_add_lattice(mcgb_ctx *ctx, double x0, double y0, double pitch, int nx, int ny,
                     const int *universes, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || nx <= 0 || ny <= 0 || !(pitch > 0.0) || !universes)
        return fail(MCGB_E_INVALID_ARG, "bad lattice");
    LatDef L{x0, y0, pitch, nx, ny, std::vector<int>(universes, universes + (size_t)nx * ny)};
    ctx->def.lats.push_back(L);
    if (id) *id = (int)ctx->def.lats.size() - 1;
    return MCGB_OK;
}

int mcgb_set_groups(mcgb_ctx *ctx, int G)
{
    if (ctx) ctx->def_version++;
    if (!ctx || G <= 0 || G > MAX_G) return fail(MCGB_E_INVALID_ARG, "bad group count");
    if (ctx->def.ce == 1 || !ctx->def.mg.empty()) return fail(MCGB_E_STATE, "groups already fixed");
    ctx->def.G = G;
    ctx->def.ce = 0;
    return MCGB_OK;
}

static int check_mg(int G, const double *st, const double *ss, const double *nf)
{
    for (int g = 0; g < G; g++) {
        if (!(st[g] >= 0.0) || !(nf[g] >= 0.0)) return fail(MCGB_E_INVALID_ARG, "negative cross section");
        double acc = 0.0;
        for (int h = 0; h < G; h++) {
            if (!(ss[g * G + h] >= 0.0)) return fail(MCGB_E_INVALID_ARG, "negative cross section");
            acc = acc + ss[g * G + h];
        }
        if (acc > st[g]) return fail(MCGB_E_INVALID_ARG, "scattering exceeds total");
    }
    return MCGB_OK;
}

int mcgb_add_material_mg(mcgb_ctx *ctx, const double *sigma_t, const double *sigma_s,
                         const double *nu_sigma_f, const double *chi, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || !sigma_t || !sigma_s || !nu_sigma_f || !chi) return fail(MCGB_E_INVALID_ARG, "null array");
    int G = ctx->def.G;
    if (ctx->def.ce != 0 || G <= 0) return fail(MCGB_E_STATE, "call mcgb_set_groups first");
    CKR(check_mg(G, sigma_t, sigma_s, nu_sigma_f));
    MatMGDef m{std::vector<double>(sigma_t, sigma_t + G), std::vector<double>(sigma_s, sigma_s + G * G),
               std::vector<double>(nu_sigma_f, nu_sigma_f + G), std::vector<double>(chi, chi + G)};
    ctx->def.mg.push_back(m);
    if (id) *id = (int)ctx->def.mg.size() - 1;
    return MCGB_OK;
}

int mcgb_update_material_mg(mcgb_ctx *ctx, int id, const double *sigma_t, const double *sigma_s,
                            const double *nu_sigma_f, const double *chi)
{
    if (ctx) ctx->def_version++;
    if (!ctx || id < 0 || id >= (int)ctx->def.mg.size()) return fail(MCGB_E_NOT_FOUND, "no such material");
    int G = ctx->def.G;
    CKR(check_mg(G, sigma_t, sigma_s, nu_sigma_f));
    MatMGDef &m = ctx->def.mg[id];
    m.sigt.assign(sigma_t, sigma_t + G);
    m.sigs.assign(sigma_s, sigma_s + G * G);
    m.nusf.assign(nu_sigma_f, nu_sigma_f + G);
    if (chi) m.chi.assign(chi, chi + G);
    return MCGB_OK;
}

int mcgb_add_nuclide_ce(mcgb_ctx *ctx, double A, int n, const double *E, const double *sig_s,
                        const double *sig_c, const double *sig_f, double nu, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || n < 2 || !(A > 0.0) || !E || !sig_s || !sig_c || !sig_f || nu < 0.0)
        return fail(MCGB_E_INVALID_ARG, "bad nuclide");
    if (ctx->def.ce == 0) return fail(MCGB_E_STATE, "problem is multigroup");
    for (int k = 1; k < n; k++)
        if (!(E[k] > E[k - 1])) return fail(MCGB_E_INVALID_ARG, "energy grid not increasing");
    for (int k = 0; k < n; k++)
        if (!(sig_s[k] >= 0.0 && sig_c[k] >= 0.0 && sig_f[k] >= 0.0))
            return fail(MCGB_E_INVALID_ARG, "negative cross section");
    ctx->def.ce = 1;
    NucDef u{A, nu, std::vector<double>(E, E + n), std::vector<double>(sig_s, sig_s + n),
             std::vector<double>(sig_c, sig_c + n), std::vector<double>(sig_f, sig_f + n)};
    ctx->def.nucs.push_back(u);
    if (id) *id = (int)ctx->def.nucs.size() - 1;
    return MCGB_OK;
}

int mcgb_add_material_ce(mcgb_ctx *ctx, int n, const int *nuclides, const double *density, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || n <= 0 || n > MAX_NUC || !nuclides || !density)
        return fail(MCGB_E_INVALID_ARG, "bad material");
    if (ctx->def.ce != 1) return fail(MCGB_E_STATE, "add nuclides first");
    MatCEDef m;
    for (int k = 0; k < n; k++) {
        if (nuclides[k] < 0 || nuclides[k] >= (int)ctx->def.nucs.size())
            return fail(MCGB_E_INVALID_ARG, "bad nuclide id");
        if (!(density[k] >= 0.0)) return fail(MCGB_E_INVALID_ARG, "negative density");
        m.nuc.push_back(nuclides[k]);
        m.dens.push_back(density[k]);
    }
    ctx->def.mce.push_back(m);
    if (id) *id = (int)ctx->def.mce.size() - 1;
    return MCGB_OK;
}

int mcgb_set_source(mcgb_ctx *ctx, int kind, const double *params, int accept, int energy_kind,
                    const double *energy, int n_energy, int dir_kind, const double *beam)
{
    if (ctx) ctx->def_version++;
    if (!ctx || !params || (kind != MCGB_SRC_BOX && kind != MCGB_SRC_POINT) || accept < 0 ||
        accept > 1 || energy_kind < 0 || energy_kind > 3 || (dir_kind != 0 && dir_kind != 1))
        return fail(MCGB_E_INVALID_ARG, "bad source");
    if ((energy_kind == MCGB_ENERGY_PDF || energy_kind == MCGB_ENERGY_FIXED) && (!energy || n_energy < 1))
        return fail(MCGB_E_INVALID_ARG, "source energy data missing");
    if (dir_kind == MCGB_DIR_BEAM && !beam) return fail(MCGB_E_INVALID_ARG, "beam direction missing");
    SrcDef s;
    s.kind = kind;
    s.accept = accept;
    s.ekind = energy_kind;
    s.dkind = dir_kind;
    std::memcpy(s.p, params, sizeof(double) * (kind == MCGB_SRC_BOX ? 6 : 3));
    if (dir_kind == MCGB_DIR_BEAM) std::memcpy(s.beam, beam, sizeof s.beam);
    if (energy_kind == MCGB_ENERGY_PDF) s.pdf.assign(energy, energy + n_energy);
    if (energy_kind == MCGB_ENERGY_FIXED) s.E = energy[0];
    ctx->def.src = s;
    return MCGB_OK;
}

int mcgb_add_tally(mcgb_ctx *ctx, int filter, int n_edges, const double *edges, int *id)
{
    if (ctx) ctx->def_version++;
    if (!ctx || filter < 0 || filter > 2 || n_edges < 0 || (n_edges > 0 && !edges))
        return fail(MCGB_E_INVALID_ARG, "bad tally");
    TallyDef t;
    t.filter = filter;
    for (int k = 0; k < n_edges; k++) {
        if (k > 0 && !(edges[k] > edges[k - 1])) return fail(MCGB_E_INVALID_ARG, "edges not increasing");
        t.edges.push_back(edges[k]);
    }
    ctx->def.tallies.push_back(t);
    if (id) *id = (int)ctx->def.tallies.size() - 1;
    return MCGB_OK;
}

int mcgb_set_max_collisions(mcgb_ctx *ctx, int max_collisions)
{
    if (ctx) ctx->def_version++;
    if (!ctx || max_collisions < 0) return fail(MCGB_E_INVALID_ARG, "bad max_collisions");
    ctx->def.max_coll = max_collisions;
    return MCGB_OK;
}

int mcgb_set_free_gas(mcgb_ctx *ctx, double kT, double cut)
{
    if (ctx) ctx->def_version++;
    if (!ctx || !(kT > 0.0) || !std::isfinite(kT) || !(cut >= 0.0) || !std::isfinite(cut))
        return fail(MCGB_E_INVALID_ARG, "bad free-gas settings");
    ctx->def.fg_kT = kT;
    ctx->def.fg_cut = cut;
    return MCGB_OK;
}

int mcgb_set_time(mcgb_ctx *ctx, double t0, double t_cut)
{
    if (ctx) ctx->def_version++;
    if (!ctx || !(t0 >= 0.0) || !(t_cut > t0) || !std::isfinite(t_cut))
        return fail(MCGB_E_INVALID_ARG, "need 0 <= t0 < t_cut < inf");
    ctx->def.time_on = true;
    ctx->def.t0 = t0;
    ctx->def.tcut = t_cut;
    return MCGB_OK;
}

int mcgb_set_inverse_speeds(mcgb_ctx *ctx, int G, const double *inv_v)
{
    if (ctx) ctx->def_version++;
    if (!ctx || G <= 0 || G != ctx->def.G || !inv_v)
        return fail(MCGB_E_INVALID_ARG, "one inverse speed per group");
    for (int g = 0; g < G; g++)
        if (!(inv_v[g] > 0.0) || !std::isfinite(inv_v[g]))
            return fail(MCGB_E_INVALID_ARG, "inverse speeds must be positive and finite");
    ctx->def.invv.assign(inv_v, inv_v + G);
    return MCGB_OK;
}

int mcgb_set_tally_time_bins(mcgb_ctx *ctx, int tally, int n_edges, const double *edges)
{
    if (ctx) ctx->def_version++;
    if (!ctx || tally < 0 || tally >= (int)ctx->def.tallies.size() || n_edges < 2 || !edges)
        return fail(MCGB_E_INVALID_ARG, "bad time bins");
    if (!(edges[0] >= 0.0)) return fail(MCGB_E_INVALID_ARG, "time edges must be >= 0");
    for (int k = 1; k < n_edges; k++)
        if (!(edges[k] > edges[k - 1]) || !std::isfinite(edges[k]))
            return fail(MCGB_E_INVALID_ARG, "time edges must increase");
    ctx->def.tallies[tally].tedges.assign(edges, edges + n_edges);
    return MCGB_OK;
}

int mcgb_run_eigenvalue(mcgb_ctx *ctx, int64_t n, int inactive, int active, uint64_t seed)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    CK(cudaSetDevice(ctx->device));
    return run_eigen(ctx, n, inactive, active, seed);
}

int mcgb_eigen_begin(mcgb_ctx *ctx, int64_t n, int inactive, int active, uint64_t seed)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    CK(cudaSetDevice(ctx->device));
    return eigen_begin(ctx, n, inactive, active, seed);
}

int mcgb_eigen_cycles(mcgb_ctx *ctx, int n_cycles)
{
    if (!ctx || n_cycles < 0) return fail(MCGB_E_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(ctx->device));
    return eigen_cycles(ctx, n_cycles);
}

int mcgb_eigen_finish(mcgb_ctx *ctx)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    CK(cudaSetDevice(ctx->device));
    return eigen_finish(ctx);
}

// ---- checkpoint and restart of a power iteration ---------------------------
namespace {

struct CkptHeader {
    char magic[8];
    uint64_t fingerprint, seed;
    int64_t N, launches;
    int32_t inactive, active, cyc, acc;
    mcgb_counters counters;
    unsigned long long cnt[8];
};
const char CKPT_MAGIC[8] = {'M', 'C', 'G', 'B', 'E', 'I', 'G', '1'};

// header | k sums [2 cyc] | bank sizes [cyc] | cycle and transport times [cyc] each |
// tally sums, sums of squares [acc] each | next cycle's sources [N] | checksum
size_t ckpt_size(int64_t cyc, int64_t acc, int64_t N)
{
    return sizeof(CkptHeader) + (size_t)cyc * (2 * sizeof(double) + sizeof(int64_t) + 2 * sizeof(double)) +
           (size_t)acc * 2 * sizeof(double) + (size_t)N * sizeof(ShardSite) + sizeof(uint64_t);
}

uint64_t ckpt_checksum(const unsigned char *p, size_t n)   // FNV-1a over 8-byte words, then the tail
{
    uint64_t h = 14695981039346656037ULL;
    const size_t nw = n / 8;
    for (size_t k = 0; k < nw; k++) {
        uint64_t w;
        std::memcpy(&w, p + 8 * k, 8);
        h = (h ^ w) * 1099511628211ULL;
    }
    for (size_t k = 8 * nw; k < n; k++) h = (h ^ (uint64_t)p[k]) * 1099511628211ULL;
    return h;
}

}  // namespace

int mcgb_eigen_checkpoint(mcgb_ctx *c, void *buf, size_t cap, size_t *needed)
{
    if (!c || !needed) return fail(MCGB_E_INVALID_ARG, "null argument");
    EigenRun &e = c->eig;
    if (!e.on) return fail(MCGB_E_STATE, "no eigenvalue run in progress");
    if (e.cyc < 1 || e.cyc >= e.ncyc) return fail(MCGB_E_STATE, "a checkpoint is taken between two cycles");
    const int acc = std::max(c->world->W.acc_size, 0);
    const int cyc = e.cyc;
    const size_t size = ckpt_size(cyc, acc, e.N);
    *needed = size;
    if (!buf) return MCGB_OK;
    if (cap < size) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, CKPT_MAGIC, 8);
    h.fingerprint = c->world->fingerprint;
    h.seed = e.seed_arg;
    h.N = e.N;
    h.launches = c->launches;
    h.inactive = e.inactive;
    h.active = e.active;
    h.cyc = cyc;
    h.acc = acc;
    h.counters = c->counters;
    unsigned char *p = static_cast<unsigned char *>(buf);
    unsigned char *q = p + sizeof h;
    CK(cudaMemcpyAsync(h.cnt, r.cnt, sizeof h.cnt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(q, r.kout, sizeof(double) * 2 * cyc, cudaMemcpyDeviceToHost, st));
    q += sizeof(double) * 2 * cyc;
    std::memcpy(q, c->cyc_m.data(), sizeof(int64_t) * cyc);
    q += sizeof(int64_t) * cyc;
    std::memcpy(q, c->cyc_ms.data(), sizeof(double) * cyc);
    q += sizeof(double) * cyc;
    std::memcpy(q, c->cyc_tms.data(), sizeof(double) * cyc);
    q += sizeof(double) * cyc;
    CK(cudaMemcpyAsync(q, r.tsum, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    q += sizeof(double) * acc;
    CK(cudaMemcpyAsync(q, r.tsum2, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    q += sizeof(double) * acc;
    // the next cycle's sources, in source order: bank sites through the resampled indices
    DevAlloc tmp;
    ShardSite *src = nullptr;
    CKR(tmp.get(src, e.N));
    launch_pack_sites(r.bank[e.cur], r.src_idx, e.N, 0, src, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(q, src, sizeof(ShardSite) * e.N, cudaMemcpyDeviceToHost, st));
    q += sizeof(ShardSite) * e.N;
    CK(cudaStreamSynchronize(st));
    std::memcpy(p, &h, sizeof h);
    const uint64_t sum = ckpt_checksum(p, size - sizeof(uint64_t));
    std::memcpy(q, &sum, sizeof sum);
    return MCGB_OK;
}

int mcgb_eigen_restore(mcgb_ctx *c, const void *buf, size_t size)
{
    if (!c || !buf) return fail(MCGB_E_INVALID_ARG, "null argument");
    if (size < sizeof(CkptHeader) + sizeof(uint64_t)) return fail(MCGB_E_INVALID_ARG, "truncated checkpoint");
    const unsigned char *p = static_cast<const unsigned char *>(buf);
    CkptHeader h;
    std::memcpy(&h, p, sizeof h);
    if (std::memcmp(h.magic, CKPT_MAGIC, 8) != 0) return fail(MCGB_E_INVALID_ARG, "not a checkpoint");
    if (h.N <= 0 || h.N > (int64_t)1 << 30 || h.inactive < 0 || h.active < 1 ||
        h.inactive + h.active > 4096 || h.cyc < 1 || h.cyc >= h.inactive + h.active || h.acc < 0 ||
        h.acc > (1 << 30))
        return fail(MCGB_E_INVALID_ARG, "bad checkpoint header");
    const size_t want = ckpt_size(h.cyc, h.acc, h.N);
    if (size != want) return fail(MCGB_E_INVALID_ARG, "truncated checkpoint");
    uint64_t sum;
    std::memcpy(&sum, p + want - sizeof sum, sizeof sum);
    if (ckpt_checksum(p, want - sizeof sum) != sum) return fail(MCGB_E_INVALID_ARG, "checkpoint checksum mismatch");
    CK(cudaSetDevice(c->device));
    CKR(eigen_begin(c, h.N, h.inactive, h.active, h.seed));
    EigenRun &e = c->eig;
    if (c->world->fingerprint != h.fingerprint || c->world->W.acc_size != h.acc) {
        e.on = false;
        return fail(MCGB_E_INVALID_ARG, "the checkpoint is of another problem");
    }
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const int cyc = h.cyc, acc = h.acc;
    const unsigned char *q = p + sizeof h;
    CK(cudaMemcpyAsync(r.cnt, h.cnt, sizeof h.cnt, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(r.kout, q, sizeof(double) * 2 * cyc, cudaMemcpyHostToDevice, st));
    q += sizeof(double) * 2 * cyc;
    std::memcpy(c->cyc_m.data(), q, sizeof(int64_t) * cyc);
    q += sizeof(int64_t) * cyc;
    std::memcpy(c->cyc_ms.data(), q, sizeof(double) * cyc);
    q += sizeof(double) * cyc;
    std::memcpy(c->cyc_tms.data(), q, sizeof(double) * cyc);
    q += sizeof(double) * cyc;
    CK(cudaMemcpyAsync(r.tsum, q, sizeof(double) * acc, cudaMemcpyHostToDevice, st));
    q += sizeof(double) * acc;
    CK(cudaMemcpyAsync(r.tsum2, q, sizeof(double) * acc, cudaMemcpyHostToDevice, st));
    q += sizeof(double) * acc;
    DevAlloc tmp;
    ShardSite *src = nullptr;
    CKR(tmp.get(src, h.N));
    CK(cudaMemcpyAsync(src, q, sizeof(ShardSite) * h.N, cudaMemcpyHostToDevice, st));
    e.cur = cyc & 1;
    launch_sites_to_bank(src, h.N, r.bank[e.cur], st);
    CK(cudaGetLastError());
    std::vector<int> iota(h.N);
    for (int64_t k = 0; k < h.N; k++) iota[k] = (int)k;
    CK(cudaMemcpyAsync(r.src_idx, iota.data(), sizeof(int) * h.N, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    e.cyc = cyc;
    c->counters = h.counters;
    c->launches = h.launches + 1;
    return MCGB_OK;
}

int mcgb_get_cycle_times(mcgb_ctx *ctx, int n_cycles, double *transport_ms, double *cycle_ms)
{
    if (!ctx || n_cycles < 0) return fail(MCGB_E_INVALID_ARG, "bad argument");
    for (int i = 0; i < n_cycles && i < (int)ctx->cyc_tms.size(); i++) {
        if (transport_ms) transport_ms[i] = ctx->cyc_tms[i];
        if (cycle_ms) cycle_ms[i] = ctx->cyc_ms[i];
    }
    return MCGB_OK;
}

int mcgb_run_fixed_source(mcgb_ctx *ctx, int64_t n, int batches, uint64_t seed)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    if (n <= 0 || batches < 1 || batches > n) return fail(MCGB_E_INVALID_ARG, "bad run size");
    CK(cudaSetDevice(ctx->device));
    CKR(build_single(ctx, n, batches, seed));
    return run_fixed_world(ctx, false, -1);
}

int mcgb_get_k(mcgb_ctx *ctx, double out[6])
{
    if (!ctx || !out) return fail(MCGB_E_INVALID_ARG, "null argument");
    std::memcpy(out, ctx->k, sizeof ctx->k);
    return MCGB_OK;
}

int mcgb_get_cycle_k(mcgb_ctx *ctx, int n_cycles, double *k_tl, double *k_col, int64_t *bank)
{
    if (!ctx || n_cycles < 0) return fail(MCGB_E_INVALID_ARG, "bad argument");
    for (int i = 0; i < n_cycles && i < (int)ctx->cyc_ktl.size(); i++) {
        if (k_tl) k_tl[i] = ctx->cyc_ktl[i];
        if (k_col) k_col[i] = ctx->cyc_kc[i];
        if (bank) bank[i] = ctx->cyc_m[i];
    }
    return MCGB_OK;
}

int mcgb_tally_size(mcgb_ctx *ctx, int tally, int *n_bins, int *n_ebins, int *n_tbins)
{
    if (!ctx || tally < 0 || tally >= (int)ctx->def.tallies.size()) return fail(MCGB_E_NOT_FOUND, "no such tally");
    const ProblemDef &d = ctx->def;
    const TallyDef &t = d.tallies[tally];
    int nmat = d.ce == 1 ? (int)d.mce.size() : (int)d.mg.size();
    int nb = t.filter == MCGB_FILTER_CELL ? (int)d.cells.size()
           : t.filter == MCGB_FILTER_LATTICE ? (d.lats.empty() ? 0 : d.lats[0].nx * d.lats[0].ny) : nmat;
    if (n_bins) *n_bins = nb;
    if (n_ebins) *n_ebins = d.ce == 1 ? (int)t.edges.size() - 1 : d.G;
    if (n_tbins) *n_tbins = t.tedges.empty() ? 1 : (int)t.tedges.size() - 1;
    return MCGB_OK;
}

int mcgb_get_tally(mcgb_ctx *ctx, int tally, double *mean, double *sd, size_t cap, size_t *needed)
{
    if (!ctx || tally < 0 || tally >= (int)ctx->t_mean.size()) return fail(MCGB_E_NOT_FOUND, "no tally results");
    size_t n = ctx->t_mean[tally].size();
    if (needed) *needed = n;
    if (cap < n) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    if (mean) std::memcpy(mean, ctx->t_mean[tally].data(), n * sizeof(double));
    if (sd) std::memcpy(sd, ctx->t_sd[tally].data(), n * sizeof(double));
    return MCGB_OK;
}

// ---------------------------------------------------------------------------
// Sharded power iteration: this context transports source indices
// [j0, j0 + n) of every cycle of an N-history power iteration.  Stream ids stay
// global (cycle 2^32 + j): the problem's first slot is given the global index
// j0 through its generation base.  Bank order, resampling and statistics are
// the caller's exchange step (the concatenation of the ranks' ordered banks in
// rank order is the global (parent, child) order).
int mcgb_shard_begin(mcgb_ctx *c, int64_t N, int64_t j0, int64_t n, int inactive, int active,
                     uint64_t seed)
{
    if (!c) return fail(MCGB_E_INVALID_ARG, "null context");
    if (N <= 0 || N > (int64_t)1 << 30 || j0 < 0 || n <= 0 || j0 + n > N)
        return fail(MCGB_E_INVALID_ARG, "bad shard");
    if (inactive < 0 || active < 1 || inactive + active > 4096)
        return fail(MCGB_E_INVALID_ARG, "bad cycle counts");
    if (c->def.time_on) return fail(MCGB_E_INVALID_ARG, "time dependence is for fixed-source runs");
    CK(cudaSetDevice(c->device));
    c->eig.on = false;
    c->shard.on = false;
    CKR(build_single(c, n, 1, seed));
    double bf = c->opts.bank_factor > 0 ? c->opts.bank_factor : 3.0;
    int64_t cap_b = (int64_t)(bf * (double)n) + 1024;
    CKR(prepare_buffers(c, std::max(n, cap_b), cap_b));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    int acc = W.acc_size;
    CK(cudaMemsetAsync(r.tacc, 0, sizeof(double) * (size_t)acc * W.nrep, st));
    CK(cudaMemsetAsync(r.tsum, 0, sizeof(double) * (size_t)std::max(acc, 1), st));
    CK(cudaMemsetAsync(r.tsum2, 0, sizeof(double) * (size_t)std::max(acc, 1), st));
    CK(cudaMemsetAsync(r.kout, 0, sizeof(double) * 2 * 4096, st));
    CK(cudaMemsetAsync(r.cnt, 0, sizeof(unsigned long long) * 8, st));
    CK(cudaMemsetAsync(r.err, 0, sizeof(int), st));
    int64_t base[2] = {-j0, n - j0};
    CK(cudaMemcpyAsync(r.gen_base[0], base, sizeof base, cudaMemcpyHostToDevice, st));
    std::vector<int> iota(n);
    for (int64_t k = 0; k < n; k++) iota[k] = (int)k;
    CK(cudaMemcpyAsync(r.src_idx, iota.data(), 4 * n, cudaMemcpyHostToDevice, st));
    c->shard.mem.release();
    CKR(c->shard.mem.get(c->shard.sums, 2 + acc));
    CK(cudaStreamSynchronize(st));
    c->counters = mcgb_counters{};
    c->counters.world_bytes = (int64_t)c->world->bytes;
    c->launches = 0;
    c->shard.on = true;
    c->shard.N = N;
    c->shard.j0 = j0;
    c->shard.n = n;
    c->shard.M = 0;
    c->shard.inactive = inactive;
    c->shard.ncyc = inactive + active;
    c->shard.cyc = 0;
    c->shard.state = 0;
    c->cyc_m.assign(inactive + active, 0);
    c->cyc_ktl.assign(inactive + active, 0.0);
    c->cyc_kc.assign(inactive + active, 0.0);
    return MCGB_OK;
}

int mcgb_shard_cycle(mcgb_ctx *c, int cycle, int64_t *m)
{
    if (!c || !c->shard.on) return fail(MCGB_E_STATE, "no shard begun");
    if (!m) return fail(MCGB_E_INVALID_ARG, "null output");
    if (cycle != c->shard.cyc || c->shard.state != 0 || cycle >= c->shard.ncyc)
        return fail(MCGB_E_STATE, "cycles run in order: transport, export, import");
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    const int64_t n = c->shard.n;
    Bank &Bs = r.bank[0], &Bd = r.bank[1];
    double *sums = c->shard.sums;
    CK(cudaMemsetAsync(r.bank_n, 0, sizeof(int), st));
    CK(cudaMemsetAsync(sums, 0, sizeof(double) * 2, st));
    RunBufs R = run_bufs(c, nullptr, -1, 0);
    CKR(transport_generation(c, R, cycle, n, r.gen_base[0], cycle > 0 ? r.src_idx : nullptr, 1, Bs,
                             Bd));
    launch_reduce_gen(r.P, n, nullptr, sums, r.cnt, st);
    scan_exclusive(r.P.nfis, r.off, n, r.M, r.scratch, st);
    launch_perm(Bd, r.off, r.M, r.perm, c->sms * 4, st);
    if (W.acc_size > 0) {
        launch_acc_reduce(r.tacc, W.acc_size, W.nrep, sums + 2, st);
        CK(cudaMemsetAsync(r.tacc, 0, sizeof(double) * (size_t)W.acc_size * W.nrep, st));
    }
    c->launches += 5;
    int64_t M;
    int err;
    CKR(read_flags(c, M, err));
    if (err & ERR_BANK_OVERFLOW)
        return fail(MCGB_E_BANK_OVERFLOW, "fission bank overflow in cycle " + std::to_string(cycle) +
                                              " (raise opts.bank_factor)");
    if (err & ERR_SOURCE) return fail(MCGB_E_STATE, "source sampling failed");
    if (err & ERR_ITER) return fail(MCGB_E_TIMEOUT, "persistent event loop pass limit reached");
    c->shard.M = M;
    c->shard.state = 1;
    *m = M;
    c->counters.histories += n;
    c->counters.generations += 1;
    CKR(fetch_counters(c));
    return MCGB_OK;
}

int mcgb_shard_export(mcgb_ctx *c, mcgb_site *bank, size_t bank_cap, double *sums, size_t sums_cap,
                      size_t *n_sums)
{
    if (!c || !c->shard.on) return fail(MCGB_E_STATE, "no shard begun");
    const size_t ns = 2 + (size_t)std::max(c->world->W.acc_size, 0);
    if (n_sums) *n_sums = ns;
    if (!sums && !bank) return MCGB_OK;   // size query
    if (c->shard.state != 1) return fail(MCGB_E_STATE, "run mcgb_shard_cycle first");
    const int64_t M = c->shard.M;
    if (bank_cap < (size_t)M || sums_cap < ns) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    if ((M > 0 && !bank) || !sums) return fail(MCGB_E_INVALID_ARG, "null output");
    CK(cudaSetDevice(c->device));
    cudaStream_t st = c->stream;
    launch_pack_sites(c->rs.bank[1], c->rs.perm, M, c->shard.j0, reinterpret_cast<ShardSite *>(bank),
                      st);
    CK(cudaMemcpyAsync(sums, c->shard.sums, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
    c->launches += 1;
    CK(cudaGetLastError());
    c->shard.state = 2;
    return MCGB_OK;
}

int mcgb_shard_import(mcgb_ctx *c, int cycle, const double *sums, const mcgb_site *bank, int64_t M)
{
    if (!c || !c->shard.on) return fail(MCGB_E_STATE, "no shard begun");
    if (cycle != c->shard.cyc || c->shard.state != 2)
        return fail(MCGB_E_STATE, "cycles run in order: transport, export, import");
    if (!sums || M < 0 || (M > 0 && !bank)) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (M == 0) {
        c->shard.on = false;
        return fail(MCGB_E_STATE, "fission bank empty after cycle " + std::to_string(cycle));
    }
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const int acc = c->world->W.acc_size;
    const double N = (double)c->shard.N;
    launch_shard_stats(sums, acc, N, cycle, cycle >= c->shard.inactive, r.kout, r.tsum, r.tsum2, st);
    c->launches += 1;
    c->cyc_m[cycle] = M;
    if (cycle + 1 < c->shard.ncyc) {
        if (c->shard.n > r.bank[0].cap) return fail(MCGB_E_BANK_OVERFLOW, "source slice above the bank");
        uint64_t rs = rng_stream(c->world->probs[0].seed, ((uint64_t)cycle << 32) + 0xFFFFFFFFULL);
        double xi = draw_host(rs);
        launch_unpack_sources(reinterpret_cast<const ShardSite *>(bank), M, c->shard.N, c->shard.j0,
                              c->shard.n, xi, r.bank[0], st);
        c->launches += 1;
    }
    CK(cudaGetLastError());
    c->shard.cyc = cycle + 1;
    c->shard.state = 0;
    return MCGB_OK;
}

// Statistics of a power iteration run in pieces (sharded or domain
// decomposed): per-cycle k from the summed estimators in r.kout, the bank
// sizes in c->cyc_m, k means and sds over the active cycles, tally batch
// means and sds from r.tsum / r.tsum2 -- as eigen_finish computes them.
static int finish_power_iteration(mcgb_ctx *c, int ncyc, int inactive, double N)
{
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const int active = ncyc - inactive;
    const int acc = c->world->W.acc_size;
    std::vector<double> kout(2 * ncyc), ts(std::max(acc, 1)), ts2(std::max(acc, 1));
    CK(cudaMemcpyAsync(kout.data(), r.kout, sizeof(double) * 2 * ncyc, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ts.data(), r.tsum, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ts2.data(), r.tsum2, sizeof(double) * acc, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double ks[3] = {0, 0, 0}, ks2[3] = {0, 0, 0};
    for (int cyc = 0; cyc < ncyc; cyc++) {
        c->cyc_ktl[cyc] = kout[2 * cyc] / N;
        c->cyc_kc[cyc] = kout[2 * cyc + 1] / N;
        if (cyc >= inactive) {
            double kv[3] = {c->cyc_ktl[cyc], c->cyc_kc[cyc], (double)c->cyc_m[cyc] / N};
            for (int q = 0; q < 3; q++) {
                ks[q] += kv[q];
                ks2[q] += kv[q] * kv[q];
            }
        }
    }
    for (int q = 0; q < 3; q++) mean_sd(ks[q], ks2[q], active, c->k[2 * q], c->k[2 * q + 1]);
    DeviceWorld &dw = *c->world;
    c->t_mean.assign(c->def.tallies.size(), {});
    c->t_sd.assign(c->def.tallies.size(), {});
    for (size_t t = 0; t < c->def.tallies.size(); t++) {
        int gt = dw.tally_first[0] + (int)t;
        int nb = dw.t_nbins[gt] * dw.t_ne[gt] * std::max(1, dw.t_ntb[gt]);
        c->t_mean[t].resize(nb);
        c->t_sd[t].resize(nb);
        for (int b = 0; b < nb; b++)
            mean_sd(ts[dw.t_off[gt] + b], ts2[dw.t_off[gt] + b], active, c->t_mean[t][b],
                    c->t_sd[t][b]);
    }
    return MCGB_OK;
}

int mcgb_shard_finish(mcgb_ctx *c)
{
    if (!c || !c->shard.on) return fail(MCGB_E_STATE, "no shard begun");
    if (c->shard.cyc < c->shard.ncyc) return fail(MCGB_E_STATE, "cycles remain to be run");
    CK(cudaSetDevice(c->device));
    c->shard.on = false;
    return finish_power_iteration(c, c->shard.ncyc, c->shard.inactive, (double)c->shard.N);
}

// ---- spatial domain decomposition ------------------------------------------
int mcgb_domain_begin(mcgb_ctx *c, int64_t N, int inactive, int active, uint64_t seed, int axis,
                      const double *cuts, int n_domains, int rank)
{
    if (!c || !cuts) return fail(MCGB_E_INVALID_ARG, "null argument");
    if (N <= 0 || N > (int64_t)1 << 30 || inactive < 0 || active < 1 || inactive + active > 4096)
        return fail(MCGB_E_INVALID_ARG, "bad run size");
    if (axis < 0 || axis > 2 || n_domains < 1 || n_domains > 1024 || rank < 0 || rank >= n_domains)
        return fail(MCGB_E_INVALID_ARG, "bad domain layout");
    if (!(cuts[0] == -HUGE_VAL) || !(cuts[n_domains] == HUGE_VAL))
        return fail(MCGB_E_INVALID_ARG, "the outer cuts must be -inf and +inf");
    for (int r = 0; r < n_domains; r++)
        if (!(cuts[r] < cuts[r + 1])) return fail(MCGB_E_INVALID_ARG, "cuts must increase");
    if (c->def.time_on) return fail(MCGB_E_INVALID_ARG, "time dependence is for fixed-source runs");
    CK(cudaSetDevice(c->device));
    c->eig.on = false;
    c->shard.on = false;
    c->dom.on = false;
    CKR(build_single(c, N, 1, seed));
    double bf = c->opts.bank_factor > 0 ? c->opts.bank_factor : 3.0;
    int64_t cap_b = (int64_t)(bf * (double)N) + 1024;
    CKR(prepare_buffers(c, std::max(N, cap_b), cap_b));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    CK(cudaMemsetAsync(r.tacc, 0, sizeof(double) * (size_t)W.acc_size * W.nrep, st));
    CK(cudaMemsetAsync(r.tsum, 0, sizeof(double) * (size_t)std::max(W.acc_size, 1), st));
    CK(cudaMemsetAsync(r.tsum2, 0, sizeof(double) * (size_t)std::max(W.acc_size, 1), st));
    CK(cudaMemsetAsync(r.kout, 0, sizeof(double) * 2 * 4096, st));
    CK(cudaMemsetAsync(r.cnt, 0, sizeof(unsigned long long) * 8, st));
    CK(cudaMemsetAsync(r.err, 0, sizeof(int), st));
    auto &d = c->dom;
    d.mem.release();
    CKR(d.mem.get(d.cuts, n_domains + 1));
    CKR(d.mem.get(d.list, N));
    CKR(d.mem.get(d.outbox, N));
    CKR(d.mem.get(d.n_list, 4));
    CKR(d.mem.get(d.n_out_dev, 4));
    CKR(d.mem.get(d.work, 4));
    CKR(d.mem.get(d.glob, cap_b));
    CK(cudaMemcpyAsync(d.cuts, cuts, sizeof(double) * (n_domains + 1), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    c->counters = mcgb_counters{};
    c->counters.world_bytes = (int64_t)c->world->bytes;
    c->launches = 0;
    d.on = true;
    d.N = N;
    d.cap = cap_b;
    d.M = 0;
    d.inactive = inactive;
    d.ncyc = inactive + active;
    d.cyc = 0;
    d.rank = rank;
    d.nd = n_domains;
    d.state = 0;
    d.cut = DomainCut{axis, cuts[rank], cuts[rank + 1]};
    c->cyc_m.assign(d.ncyc, 0);
    c->cyc_ktl.assign(d.ncyc, 0.0);
    c->cyc_kc.assign(d.ncyc, 0.0);
    return MCGB_OK;
}

static int domain_check(mcgb_ctx *c, int state, const char *what)
{
    if (!c || !c->dom.on) return fail(MCGB_E_STATE, "no domain run begun");
    if (c->dom.state != state) return fail(MCGB_E_STATE, std::string("out of order: ") + what);
    return MCGB_OK;
}

int mcgb_domain_sources(mcgb_ctx *c, int cycle, const mcgb_site *bank, int64_t M)
{
    CKR(domain_check(c, 0, "sources begin a cycle"));
    auto &d = c->dom;
    if (cycle != d.cyc || cycle >= d.ncyc) return fail(MCGB_E_STATE, "cycles run in order");
    const ShardSite *b = reinterpret_cast<const ShardSite *>(bank);
    if (cycle > 0 && !b) {
        b = d.glob;   // the bank this context assembled at the last import
        M = d.M;
    }
    if (cycle > 0 && M <= 0) return fail(MCGB_E_INVALID_ARG, "no bank to resample");
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    double xi = 0.0;
    if (cycle > 0) {
        uint64_t rs = rng_stream(c->world->probs[0].seed, ((uint64_t)(cycle - 1) << 32) + 0xFFFFFFFFULL);
        xi = draw_host(rs);
    }
    CK(cudaMemsetAsync(d.n_list, 0, sizeof(int), st));
    CK(cudaMemsetAsync(r.bank_n, 0, sizeof(int), st));
    launch_dom_sources(c->world->W, r.P, cycle, d.N, cycle > 0 ? b : nullptr, M, xi, d.cut, d.cuts,
                       d.nd, d.rank, d.list, d.n_list, r.err, st);
    c->launches += 1;
    CK(cudaGetLastError());
    d.state = 1;
    return MCGB_OK;
}

int mcgb_domain_sweep(mcgb_ctx *c, int64_t *n_out)
{
    CKR(domain_check(c, 1, "sweeps follow the sources"));
    if (!n_out) return fail(MCGB_E_INVALID_ARG, "null output");
    auto &d = c->dom;
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(r.pinned + 8, d.n_list, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int n = r.pinned[8];
    CK(cudaMemsetAsync(d.n_out_dev, 0, sizeof(int), st));
    CK(cudaMemsetAsync(d.work, 0, sizeof(int), st));
    RunBufs R = run_bufs(c, nullptr, -1, 0);
    launch_dom_sweep(c->world->W, r.P, r.bank[1], R, d.list, n, d.work, d.cut, d.outbox, d.n_out_dev,
                     c->sms * 8, st);
    c->launches += n > 0 ? 1 : 0;
    CK(cudaMemsetAsync(d.n_list, 0, sizeof(int), st));
    CK(cudaMemcpyAsync(r.pinned + 9, d.n_out_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(r.pinned + 10, r.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(r.pinned + 11, r.bank_n, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int err = r.pinned[10];
    if (r.pinned[11] > r.bank[1].cap) err |= ERR_BANK_OVERFLOW;
    if (err & ERR_BANK_OVERFLOW)
        return fail(MCGB_E_BANK_OVERFLOW, "fission bank overflow (raise opts.bank_factor)");
    if (err & ERR_SOURCE) return fail(MCGB_E_STATE, "source sampling failed");
    d.n_out = r.pinned[9];
    *n_out = d.n_out;
    return MCGB_OK;
}

int mcgb_domain_outbox(mcgb_ctx *c, mcgb_flight *out, size_t cap)
{
    CKR(domain_check(c, 1, "the outbox follows a sweep"));
    auto &d = c->dom;
    if (cap < (size_t)d.n_out || (d.n_out > 0 && !out))
        return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    CK(cudaSetDevice(c->device));
    launch_dom_pack(c->rs.P, d.outbox, (int)d.n_out, d.cut, d.rank, reinterpret_cast<FlightRec *>(out),
                    c->stream);
    c->launches += d.n_out > 0 ? 1 : 0;
    CK(cudaGetLastError());
    return MCGB_OK;
}

int mcgb_domain_inbox(mcgb_ctx *c, const mcgb_flight *in, int64_t n)
{
    CKR(domain_check(c, 1, "the inbox follows a sweep"));
    if (n < 0 || (n > 0 && !in)) return fail(MCGB_E_INVALID_ARG, "bad inbox");
    CK(cudaSetDevice(c->device));
    auto &d = c->dom;
    launch_dom_unpack(c->world->W, c->rs.P, reinterpret_cast<const FlightRec *>(in), n, d.rank,
                      d.list, d.n_list, c->stream);
    c->launches += n > 0 ? 1 : 0;
    CK(cudaGetLastError());
    return MCGB_OK;
}

int mcgb_domain_export(mcgb_ctx *c, int32_t *nfis, mcgb_site *sites, size_t sites_cap, double *sums,
                       size_t sums_cap, size_t *m, size_t *n_sums)
{
    CKR(domain_check(c, 1, "the export ends a cycle's sweeps"));
    auto &d = c->dom;
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    const size_t ns = 2 + (size_t)std::max(W.acc_size, 0);
    CK(cudaMemcpyAsync(r.pinned + 11, r.bank_n, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t mloc = r.pinned[11];
    if (m) *m = (size_t)mloc;
    if (n_sums) *n_sums = ns;
    if (!nfis && !sites && !sums) return MCGB_OK;   // size query
    if (!nfis || !sums || (mloc > 0 && !sites)) return fail(MCGB_E_INVALID_ARG, "null output");
    if (sites_cap < (size_t)mloc || sums_cap < ns) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    CK(cudaMemsetAsync(sums, 0, sizeof(double) * 2, st));
    launch_dom_reduce(r.P, d.N, sums, r.cnt, nfis, st);
    if (W.acc_size > 0) {
        launch_acc_reduce(r.tacc, W.acc_size, W.nrep, sums + 2, st);
        CK(cudaMemsetAsync(r.tacc, 0, sizeof(double) * (size_t)W.acc_size * W.nrep, st));
    }
    launch_dom_sites(r.bank[1], mloc, reinterpret_cast<ShardSite *>(sites), st);
    c->launches += 3;
    CK(cudaGetLastError());
    d.state = 2;
    return MCGB_OK;
}

int mcgb_domain_import(mcgb_ctx *c, int cycle, const double *sums, const int32_t *nfis,
                       const mcgb_site *sites, int64_t M)
{
    CKR(domain_check(c, 2, "the import follows the export"));
    auto &d = c->dom;
    if (cycle != d.cyc) return fail(MCGB_E_STATE, "cycles run in order");
    if (!sums || !nfis || M < 0 || (M > 0 && !sites)) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (M == 0) {
        d.on = false;
        return fail(MCGB_E_STATE, "fission bank empty after cycle " + std::to_string(cycle));
    }
    if (M > d.cap) {
        d.on = false;
        return fail(MCGB_E_BANK_OVERFLOW, "fission bank overflow (raise opts.bank_factor)");
    }
    CK(cudaSetDevice(c->device));
    RunState &r = c->rs;
    cudaStream_t st = c->stream;
    const World &W = c->world->W;
    launch_shard_stats(sums, W.acc_size, (double)d.N, cycle, cycle >= d.inactive, r.kout, r.tsum,
                       r.tsum2, st);
    scan_exclusive(nfis, r.off, d.N, r.M, r.scratch, st);
    CK(cudaMemsetAsync(r.err, 0, sizeof(int), st));
    launch_dom_place(reinterpret_cast<const ShardSite *>(sites), M, r.off, d.glob, d.cap, r.err, st);
    c->launches += 5;
    CK(cudaMemcpyAsync(r.pinned + 4, r.M, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(r.pinned + 5, r.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((int64_t)r.pinned[4] != M || (r.pinned[5] & ERR_BANK_OVERFLOW)) {
        d.on = false;
        return fail(MCGB_E_STATE, "the sites do not match the histories' site counts");
    }
    c->cyc_m[cycle] = M;
    d.M = M;
    d.cyc = cycle + 1;
    d.state = 0;
    c->counters.generations += 1;
    return MCGB_OK;
}

int mcgb_domain_finish(mcgb_ctx *c)
{
    if (!c || !c->dom.on) return fail(MCGB_E_STATE, "no domain run begun");
    if (c->dom.cyc < c->dom.ncyc || c->dom.state != 0) return fail(MCGB_E_STATE, "cycles remain to be run");
    CK(cudaSetDevice(c->device));
    c->dom.on = false;
    CKR(fetch_counters(c));
    c->counters.histories = c->dom.N * c->dom.ncyc;
    return finish_power_iteration(c, c->dom.ncyc, c->dom.inactive, (double)c->dom.N);
}

int mcgb_domain_records(mcgb_ctx *c, int32_t *n_coll, int32_t *n_cross, int32_t *n_fis, int32_t *fate,
                        int32_t *g_end, uint64_t *rng_end)
{
    if (!c || !c->world || c->dom.N <= 0) return fail(MCGB_E_STATE, "no domain run");
    if (!n_coll || !n_cross || !n_fis || !fate || !g_end || !rng_end)
        return fail(MCGB_E_INVALID_ARG, "null output");
    CK(cudaSetDevice(c->device));
    launch_dom_records(c->rs.P, c->dom.N, n_coll, n_cross, n_fis, fate, g_end,
                       reinterpret_cast<unsigned long long *>(rng_end), c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return MCGB_OK;
}

int mcgb_get_counters(mcgb_ctx *ctx, mcgb_counters *out)
{
    if (!ctx || !out) return fail(MCGB_E_INVALID_ARG, "null argument");
    ctx->counters.kernel_launches = ctx->launches;
    *out = ctx->counters;
    return MCGB_OK;
}

int mcgb_get_histories(mcgb_ctx *ctx, size_t cap, int32_t *n_coll, int32_t *n_cross,
                       uint64_t *rng_end, int32_t *n_fis, int32_t *fate, int32_t *g_end,
                       size_t *needed)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    size_t n = ctx->h_coll.size();
    if (needed) *needed = n;
    if (cap < n) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    if (n_coll) std::memcpy(n_coll, ctx->h_coll.data(), n * 4);
    if (n_cross) std::memcpy(n_cross, ctx->h_cross.data(), n * 4);
    if (rng_end) std::memcpy(rng_end, ctx->h_rng.data(), n * 8);
    if (n_fis) std::memcpy(n_fis, ctx->h_fis.data(), n * 4);
    if (fate) std::memcpy(fate, ctx->h_fate.data(), n * 4);
    if (g_end) std::memcpy(g_end, ctx->h_g.data(), n * 4);
    return MCGB_OK;
}

int mcgb_get_bank(mcgb_ctx *ctx, size_t cap, double *xyz, int64_t *parent, int32_t *child,
                  int32_t *mat, size_t *needed)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    size_t n = ctx->b_parent.size();
    if (needed) *needed = n;
    if (cap < n) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    if (xyz) std::memcpy(xyz, ctx->b_xyz.data(), n * 24);
    if (parent) std::memcpy(parent, ctx->b_parent.data(), n * 8);
    if (child) std::memcpy(child, ctx->b_child.data(), n * 4);
    if (mat) std::memcpy(mat, ctx->b_mat.data(), n * 4);
    return MCGB_OK;
}

int mcgb_forward_fixed(mcgb_ctx *ctx, int64_t n, uint64_t seed, int det_cell, double *tally_out)
{
    if (!ctx || n <= 0) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (ctx->def.ce != 0) return fail(MCGB_E_STATE, "derivatives are multigroup only");
    if (ctx->def.time_on) return fail(MCGB_E_STATE, "derivatives are for time-independent runs");
    if (det_cell < 0 || det_cell >= (int)ctx->def.cells.size()) return fail(MCGB_E_INVALID_ARG, "bad detector cell");
    CK(cudaSetDevice(ctx->device));
    CKR(build_single(ctx, n, 1, seed));
    CKR(run_fixed_world(ctx, true, det_cell));
    if (tally_out) {
        int G = ctx->def.G;
        std::vector<double> acc(G, 0.0);
        // the detector tally per group: sum of the stored own tallies of all generations
        for (auto &g : ctx->grad_gens) {
            std::vector<double> own(g.n * G);
            CK(cudaMemcpy(own.data(), g.own, sizeof(double) * g.n * G, cudaMemcpyDeviceToHost));
            for (int64_t j = 0; j < g.n; j++)
                for (int q = 0; q < G; q++) acc[q] += own[j * G + q];
        }
        for (int q = 0; q < G; q++) tally_out[q] = acc[q] / (double)n;
    }
    return MCGB_OK;
}

// The replay backward on the context's stream: weights w [G] and the summed
// scores grad [nm G (G + 2)] are device buffers (grad zeroed here).
static int backward_core(mcgb_ctx *ctx, const double *w, double *grad, DevAlloc &tmp)
{
    int G = ctx->def.G, nm = (int)ctx->def.mg.size();
    int npar = nm * G * (G + 2);
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(grad, 0, sizeof(double) * npar, st));
    auto &gens = ctx->grad_gens;
    int ng = (int)gens.size();
    std::vector<double *> sub(ng, nullptr);
    for (int g = 0; g < ng; g++) CKR(tmp.get(sub[g], gens[g].n));
    for (int g = ng - 1; g >= 0; g--) {
        launch_subtree(gens[g].own, w, G, gens[g].n, g + 1 < ng ? sub[g + 1] : nullptr, gens[g].off,
                       gens[g].nfis, sub[g], st);
        ctx->launches++;
    }
    for (int g = 0; g < ng; g++) {
        ReplayArgs a{};
        a.gen = g;
        a.n = gens[g].n;
        a.site = g > 0 ? gens[g - 1].perm : nullptr;
        a.bank = g > 0 ? &gens[g - 1].bank : nullptr;
        a.own = gens[g].own;
        a.w = w;
        a.sub_next = g + 1 < ng ? sub[g + 1] : nullptr;
        a.off = gens[g].off;
        a.nfis = gens[g].nfis;
        a.det_cell = ctx->grad_cell;
        a.G = G;
        a.nmat = nm;
        a.grad = grad;
        launch_replay(ctx->world->W, a, 256, st);
        ctx->launches++;
    }
    CK(cudaGetLastError());
    return MCGB_OK;
}

int mcgb_backward_fixed(mcgb_ctx *ctx, const double *weights, double *d_sigt, double *d_sigs,
                        double *d_nusf)
{
    if (!ctx || !weights) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (!ctx->grad_ready) return fail(MCGB_E_STATE, "run mcgb_forward_fixed first");
    CK(cudaSetDevice(ctx->device));
    int G = ctx->def.G, nm = (int)ctx->def.mg.size();
    int npar = nm * G * (G + 2);
    cudaStream_t st = ctx->stream;
    DevAlloc tmp;
    double *w, *grad;
    CKR(tmp.get(w, G));
    CKR(tmp.get(grad, npar));
    CK(cudaMemcpyAsync(w, weights, sizeof(double) * G, cudaMemcpyHostToDevice, st));
    CKR(backward_core(ctx, w, grad, tmp));
    std::vector<double> h(npar);
    CK(cudaMemcpyAsync(h.data(), grad, sizeof(double) * npar, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double N = (double)ctx->grad_n;
    for (int k = 0; k < nm * G; k++) d_sigt[k] = h[k] / N;
    for (int k = 0; k < nm * G * G; k++) d_sigs[k] = h[nm * G + k] / N;
    for (int k = 0; k < nm * G; k++) d_nusf[k] = h[nm * G + nm * G * G + k] / N;
    return MCGB_OK;
}

// ---- device-pointer variants of the derivative path -----------------------
int mcgb_update_material_mg_dev(mcgb_ctx *ctx, int first, int n_mat, const double *sigma_t,
                                const double *sigma_s, const double *nu_sigma_f)
{
    if (!ctx || !sigma_t || !sigma_s || !nu_sigma_f) return fail(MCGB_E_INVALID_ARG, "null array");
    if (ctx->def.ce != 0 || ctx->def.G <= 0) return fail(MCGB_E_STATE, "problem is not multigroup");
    if (first < 0 || n_mat < 1 || first + n_mat > (int)ctx->def.mg.size())
        return fail(MCGB_E_NOT_FOUND, "no such material");
    CK(cudaSetDevice(ctx->device));
    // the tables live in the device world: build it from the definition first
    if (!ctx->world || ctx->world_version != ctx->def_version || ctx->world->probs.size() != 1)
        CKR(build_single(ctx, 1, 1, 1));
    if (!ctx->upd_bad) {
        CKR(ctx->upd_mem.get(ctx->upd_bad, 1));
        CK(cudaMemsetAsync(ctx->upd_bad, 0, sizeof(int), ctx->stream));
    }
    launch_update_mg(ctx->world->W, ctx->world->probs[0].mat0 + first, n_mat, ctx->def.G, sigma_t,
                     sigma_s, nu_sigma_f, ctx->upd_bad, ctx->stream);
    ctx->launches += 2;
    CK(cudaGetLastError());
    ctx->upd_pending = true;
    return MCGB_OK;
}

// The world of the next single-problem run of n histories from `seed`: the
// current one, with its run parameters replaced, when it was built from the
// current definition for one problem with one tally batch (it may hold device
// updates); otherwise rebuilt from the definition.
static int world_for_run(mcgb_ctx *ctx, int64_t n, uint64_t seed)
{
    DeviceWorld *dw = ctx->world.get();
    bool reuse = dw && ctx->world_version == ctx->def_version && dw->probs.size() == 1 &&
                 dw->probs[0].batches == 1;
    if (!reuse) return build_single(ctx, n, 1, seed);
    ProblemDev &P = dw->probs[0];
    P.n = n;
    P.seed = seed & 0x7FFFFFFFFFFFFFFFULL;
    CK(cudaMemcpyAsync(const_cast<ProblemDev *>(dw->W.prob), &P, sizeof(ProblemDev),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));   // P is pageable host memory
    return MCGB_OK;
}

int mcgb_forward_fixed_dev(mcgb_ctx *ctx, int64_t n, uint64_t seed, int det_cell, double *tally)
{
    if (!ctx || n <= 0) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (ctx->def.ce != 0) return fail(MCGB_E_STATE, "derivatives are multigroup only");
    if (ctx->def.time_on) return fail(MCGB_E_STATE, "derivatives are for time-independent runs");
    if (det_cell < 0 || det_cell >= (int)ctx->def.cells.size())
        return fail(MCGB_E_INVALID_ARG, "bad detector cell");
    CK(cudaSetDevice(ctx->device));
    CKR(world_for_run(ctx, n, seed));
    if (ctx->upd_pending) {
        int bad = 0;
        CK(cudaMemcpyAsync(&bad, ctx->upd_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->upd_pending = false;
        if (bad) {
            CK(cudaMemsetAsync(ctx->upd_bad, 0, sizeof(int), ctx->stream));
            return fail(MCGB_E_INVALID_ARG,
                        "mcgb_update_material_mg_dev: negative cross section or scattering above total");
        }
    }
    CKR(run_fixed_world(ctx, true, det_cell));
    if (tally) {
        int G = ctx->def.G;
        for (size_t g = 0; g < ctx->grad_gens.size(); g++) {
            launch_own_sum(ctx->grad_gens[g].own, ctx->grad_gens[g].n, G, g > 0 ? 1 : 0, tally,
                           ctx->stream);
            ctx->launches++;
        }
        if (ctx->grad_gens.empty()) CK(cudaMemsetAsync(tally, 0, sizeof(double) * G, ctx->stream));
        launch_scale(tally, G, (double)n, tally, ctx->stream);
        ctx->launches++;
        CK(cudaGetLastError());
    }
    return MCGB_OK;
}

int mcgb_backward_fixed_dev(mcgb_ctx *ctx, const double *weights, double *d_sigt, double *d_sigs,
                            double *d_nusf)
{
    if (!ctx || !weights || !d_sigt || !d_sigs || !d_nusf) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (!ctx->grad_ready) return fail(MCGB_E_STATE, "run a forward pass first");
    CK(cudaSetDevice(ctx->device));
    int G = ctx->def.G, nm = (int)ctx->def.mg.size();
    int npar = nm * G * (G + 2);
    DevAlloc tmp;
    double *grad;
    CKR(tmp.get(grad, npar));
    CKR(backward_core(ctx, weights, grad, tmp));
    double N = (double)ctx->grad_n;
    launch_scale(grad, (int64_t)nm * G, N, d_sigt, ctx->stream);
    launch_scale(grad + nm * G, (int64_t)nm * G * G, N, d_sigs, ctx->stream);
    launch_scale(grad + nm * G + nm * G * G, (int64_t)nm * G, N, d_nusf, ctx->stream);
    ctx->launches += 3;
    CK(cudaGetLastError());
    // the scratch is released when this call returns: finish with it first
    CK(cudaStreamSynchronize(ctx->stream));
    return MCGB_OK;
}

// ---- building blocks -------------------------------------------------------
int mcgb_rng_states(mcgb_ctx *ctx, uint64_t seed, uint64_t first_id, int64_t n_streams, int n_draws,
                    uint64_t *out)
{
    if (!ctx || !out || n_streams < 0 || n_draws < 1) return fail(MCGB_E_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(ctx->device));
    DevAlloc tmp;
    uint64_t *d;
    CKR(tmp.get(d, n_streams * n_draws));
    launch_rng_states(seed & LCG_MASK, first_id, n_streams, n_draws, d, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, d, sizeof(uint64_t) * n_streams * n_draws, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MCGB_OK;
}

static int ensure_world(mcgb_ctx *ctx)
{
    if (!ctx->world) {
        ctx->world.reset(new DeviceWorld());
        // a world with only the log tables when no problem is defined yet
        if (ctx->def.check().empty()) return build_single(ctx, 1, 1, 1);
        ProblemDef tiny;
        tiny.ce = 0;
        tiny.G = 1;
        tiny.s_type = {SURF_PX};
        tiny.s_bc = {BC_NONE};
        tiny.s_coef = {0, 0, 0, 0};
        tiny.cells.push_back(CellDef{0, FILL_MAT, 0, {}, {}});
        tiny.mg.push_back(MatMGDef{{1.0}, {0.0}, {0.0}, {0.0}});
        tiny.src.kind = SRC_POINT;
        std::vector<ProblemRun> runs{{&tiny, 1, 1, 1}};
        std::string e = build_world(runs, *ctx->world, ctx->stream);
        if (!e.empty()) return fail(MCGB_E_STATE, e);
        ctx->world->probs.clear();   // marks the tables as not belonging to the user's problem
        return MCGB_OK;
    }
    return MCGB_OK;
}

int mcgb_log(mcgb_ctx *ctx, int64_t n, const double *xi, double *out)
{
    if (!ctx || n < 0 || (n > 0 && (!xi || !out))) return fail(MCGB_E_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(ctx->device));
    CKR(ensure_world(ctx));
    DevAlloc tmp;
    double *dx, *dy;
    CKR(tmp.get(dx, n));
    CKR(tmp.get(dy, n));
    CK(cudaMemcpyAsync(dx, xi, 8 * n, cudaMemcpyHostToDevice, ctx->stream));
    launch_log(ctx->world->W, n, dx, dy, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dy, 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MCGB_OK;
}

int mcgb_fpint_ops(mcgb_ctx *ctx, int64_t n, const double *a, const double *b, double *out)
{
    if (!ctx || n < 0 || n > ((int64_t)1 << 31) || (n > 0 && (!a || !b || !out)))
        return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (n == 0) return MCGB_OK;
    CK(cudaSetDevice(ctx->device));
    DevAlloc tmp;
    double *da, *db, *dout;
    CKR(tmp.get(da, n));
    CKR(tmp.get(db, n));
    CKR(tmp.get(dout, 3 * n));
    CK(cudaMemcpyAsync(da, a, 8 * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(db, b, 8 * n, cudaMemcpyHostToDevice, ctx->stream));
    launch_fpint_ops(n, da, db, dout, ctx->stream);
    CK(cudaGetLastError());
    ctx->launches += 1;
    CK(cudaMemcpyAsync(out, dout, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MCGB_OK;
}

int mcgb_fp64_throughput(mcgb_ctx *ctx, int64_t iters, double *ops_per_s, double *ms)
{
    if (!ctx || iters <= 0 || !ops_per_s || !ms) return fail(MCGB_E_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(ctx->device));
    int grid = ctx->sms * 8;
    DevAlloc tmp;
    double *sink;
    CKR(tmp.get(sink, grid));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    launch_fp64_rate(grid, (long long)iters, sink, ctx->stream);
    cudaEventRecord(e0, ctx->stream);
    launch_fp64_rate(grid, (long long)iters, sink, ctx->stream);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t err = cudaStreamSynchronize(ctx->stream);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(err);
    ctx->launches += 2;
    *ms = t;
    *ops_per_s = (double)grid * 256.0 * (double)iters * fp64_rate_chains() / (t / 1e3);
    return MCGB_OK;
}

int mcgb_probe(mcgb_ctx *ctx, int64_t n, const double *pos, const double *dir, int32_t *path,
               double *dist, int32_t *kind)
{
    if (!ctx || n < 0 || (n > 0 && (!pos || !dir || !path || !dist || !kind)))
        return fail(MCGB_E_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(ctx->device));
    std::string e = ctx->def.check();
    if (!e.empty()) return fail(MCGB_E_STATE, e);
    CKR(build_single(ctx, 1, 1, 1));
    DevAlloc tmp;
    double *dp, *dd, *ddist;
    int *dpath, *dkind;
    CKR(tmp.get(dp, 3 * n)); CKR(tmp.get(dd, 3 * n)); CKR(tmp.get(ddist, n));
    CKR(tmp.get(dpath, 5 * n)); CKR(tmp.get(dkind, n));
    CK(cudaMemcpyAsync(dp, pos, 24 * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dd, dir, 24 * n, cudaMemcpyHostToDevice, ctx->stream));
    launch_probe(ctx->world->W, ctx->world->probs[0].root_univ, n, dp, dd, dpath, ddist, dkind,
                 ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(path, dpath, 20 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(dist, ddist, 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(kind, dkind, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MCGB_OK;
}

int mcgb_ce_lookup(mcgb_ctx *ctx, int mat, int64_t n, const double *E, double *out)
{
    if (!ctx || n < 0 || (n > 0 && (!E || !out))) return fail(MCGB_E_INVALID_ARG, "bad argument");
    if (ctx->def.ce != 1 || mat < 0 || mat >= (int)ctx->def.mce.size())
        return fail(MCGB_E_INVALID_ARG, "bad material");
    CK(cudaSetDevice(ctx->device));
    std::string e = ctx->def.check();
    if (!e.empty()) return fail(MCGB_E_STATE, e);
    CKR(build_single(ctx, 1, 1, 1));
    DevAlloc tmp;
    double *dE, *dout;
    CKR(tmp.get(dE, n));
    CKR(tmp.get(dout, 4 * n));
    CK(cudaMemcpyAsync(dE, E, 8 * n, cudaMemcpyHostToDevice, ctx->stream));
    launch_ce_lookup(ctx->world->W, mat, n, dE, dout, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dout, 32 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MCGB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batching: many independent fixed-source problems flattened into one world
// and run generation by generation, every problem's particles in one launch.
#include <chrono>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace {

std::mutex g_tune_mu;
std::map<std::string, mcgb_tune> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_signature(mcgb_batch *b)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, b->device);
    std::ostringstream s;
    // kernel generation: a tuning taken on other kernel builds does not apply
    s << "kv2|" << prop.name << "|sm" << prop.multiProcessorCount << "|p" << b->runs.size();
    int64_t n = 0, cells = 0, surfs = 0, groups = 0;
    for (auto &r : b->runs) {
        n += r.n;
        cells += (int64_t)r.def->cells.size();
        surfs += (int64_t)r.def->s_type.size();
        groups += r.def->G;
    }
    s << "|n" << n << "|c" << cells << "|s" << surfs << "|g" << groups;
    return s.str();
}

void tune_cache_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("MCGB_TUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string key;
        mcgb_tune t{};
        if (std::getline(is, key, '\t') && (is >> t.block >> t.blocks_per_sm >> t.pool >> t.ms))
            g_tune_cache[key] = t;
    }
}

void tune_cache_store(const std::string &key, const mcgb_tune &t)
{
    g_tune_cache[key] = t;
    const char *path = std::getenv("MCGB_TUNE_CACHE");
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << key << '\t' << t.block << ' ' << t.blocks_per_sm << ' ' << t.pool << ' ' << t.ms << '\n';
}

}  // namespace

static int batch_engine(mcgb_batch *b)
{
    if (!b->engine) {
        mcgb_ctx *c = nullptr;
        mcgb_opts o = b->opts;
        if (o.mode == 0 && o.block == 0) o.mode = MCGB_MODE_PERSISTENT;
        CKR(mcgb_create(&c, &o));
        b->engine.reset(c);
    }
    return MCGB_OK;
}

static int batch_run_runs(mcgb_batch *b, const std::vector<ProblemRun> &runs, const mcgb_tune *tune)
{
    CKR(batch_engine(b));
    mcgb_ctx *c = b->engine.get();
    CK(cudaSetDevice(c->device));
    if (tune) {
        c->opts.block = tune->block > 0 ? tune->block : c->opts.block;
        c->opts.blocks_per_sm = tune->blocks_per_sm;
        c->opts.pool = tune->pool;
    }
    if (!c->world) c->world.reset(new DeviceWorld());
    std::string e = build_world(runs, *c->world, c->stream);
    if (!e.empty()) return fail(MCGB_E_STATE, e);
    return run_fixed_world(c, false, -1);
}

extern "C" {

int mcgb_batch_create(mcgb_batch **out, const mcgb_opts *opts)
{
    if (!out) return fail(MCGB_E_INVALID_ARG, "null output");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(MCGB_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    std::unique_ptr<mcgb_batch> b(new mcgb_batch());
    if (opts) b->opts = *opts;
    if (b->opts.device < 0 || b->opts.device >= ndev) return fail(MCGB_E_INVALID_ARG, "bad device");
    b->device = b->opts.device;
    *out = b.release();
    return MCGB_OK;
}

int mcgb_batch_destroy(mcgb_batch *b)
{
    if (!b) return MCGB_OK;
    if (b->engine) {
        mcgb_destroy(b->engine.release());
    }
    delete b;
    return MCGB_OK;
}

int mcgb_batch_add_problem(mcgb_batch *b, mcgb_ctx *problem, int64_t n, int batches, uint64_t seed,
                           int *id)
{
    if (!b || !problem || n <= 0 || batches < 1 || batches > n)
        return fail(MCGB_E_INVALID_ARG, "bad argument");
    if ((int)b->runs.size() >= 4096) return fail(MCGB_E_INVALID_ARG, "at most 4096 problems");
    std::string e = problem->def.check();
    if (!e.empty()) return fail(MCGB_E_STATE, e);
    b->defs.emplace_back(new ProblemDef(problem->def));
    b->runs.push_back(ProblemRun{b->defs.back().get(), n, batches, seed});
    if (id) *id = (int)b->runs.size() - 1;
    return MCGB_OK;
}

int mcgb_batch_autotune(mcgb_batch *b, int budget_ms, mcgb_tune *out)
{
    if (!b || b->runs.empty()) return fail(MCGB_E_STATE, "empty batch");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    std::string key = tune_signature(b);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
        b->tuned = it->second;
        b->has_tune = true;
        if (out) *out = b->tuned;
        return MCGB_OK;
    }
    CKR(batch_engine(b));
    // tuning runs: every problem at 1/scale of its size (at least 64 histories)
    int64_t total = 0;
    for (auto &r : b->runs) total += r.n;
    int64_t scale = std::max<int64_t>(1, total / 400000);
    std::vector<ProblemRun> small;
    for (auto &r : b->runs) {
        ProblemRun s = r;
        s.n = std::max<int64_t>(64, r.n / scale);
        s.batches = 1;
        small.push_back(s);
    }
    mcgb_tune best{};
    best.ms = 1e30;
    auto t_start = std::chrono::steady_clock::now();
    // candidates: block-sorted pools (particles per block x resident blocks per SM)
    // and the register-resident variant (threads per block x blocks per SM)
    std::vector<mcgb_tune> cand;
    bool ce = false;
    for (auto &r : b->runs) ce = ce || r.def->ce == 1;
    for (int pool : {512, 2256, 256, 2512, 64, 128}) {
        int occ = std::max(1, pool_max_blocks_per_sm(pool, ce));
        for (int bps = occ; bps >= 1; bps = bps > 2 ? bps / 2 : bps - 1) cand.push_back({0, bps, pool, 0.0});
    }
    for (int blk : {128, 256}) {
        int occ = std::max(1, persistent_max_blocks_per_sm(blk));
        cand.push_back({blk, occ, -1, 0.0});
    }
    // device time of one batch run with tuning t
    auto timed = [&](const std::vector<ProblemRun> &runs, const mcgb_tune &t, float &ms) -> int {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, b->engine->stream));
        int r = batch_run_runs(b, runs, &t);
        CK(cudaEventRecord(e1, b->engine->stream));
        CK(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
    };
    // stage 1: every candidate on the scaled-down batch (one warm-up, one timed)
    std::vector<mcgb_tune> tried;
    for (const mcgb_tune &t : cand) {
        CKR(batch_run_runs(b, small, &t));
        float ms = 0.f;
        CKR(timed(small, t, ms));
        mcgb_tune tt = t;
        tt.ms = ms;
        tried.push_back(tt);
        double spent = std::chrono::duration<double, std::milli>(
                           std::chrono::steady_clock::now() - t_start).count();
        if (budget_ms > 0 && spent > budget_ms) break;
    }
    // stage 2: the three fastest again at full size (small runs rank the
    // launch shapes only roughly), best of those
    std::sort(tried.begin(), tried.end(),
              [](const mcgb_tune &a, const mcgb_tune &c2) { return a.ms < c2.ms; });
    if (tried.size() > 3) tried.resize(3);
    for (const mcgb_tune &t : tried) {
        float ms = 0.f;
        if (scale > 1) CKR(timed(b->runs, t, ms));
        else ms = (float)t.ms;
        if (ms < best.ms) {
            best = t;
            best.ms = ms;
        }
    }
    tune_cache_store(key, best);
    b->tuned = best;
    b->has_tune = true;
    if (out) *out = best;
    return MCGB_OK;
}

int mcgb_get_event_timing(mcgb_ctx *ctx, double *advance_ms, int64_t *particles,
                          int64_t *launches, double *bytes_per_particle)
{
    if (!ctx) return fail(MCGB_E_INVALID_ARG, "null context");
    if (!ctx->world) return fail(MCGB_E_STATE, "no problem has run");
    if (advance_ms) *advance_ms = ctx->adv_ms;
    if (particles) *particles = ctx->adv_n;
    if (launches) *launches = ctx->adv_launches;
    if (bytes_per_particle) *bytes_per_particle = event_advance_bytes(ctx->world->W);
    return MCGB_OK;
}

int mcgb_batch_run(mcgb_batch *b, const mcgb_tune *tune)
{
    if (!b || b->runs.empty()) return fail(MCGB_E_STATE, "empty batch");
    const mcgb_tune *t = tune ? tune : (b->has_tune ? &b->tuned : nullptr);
    CKR(batch_run_runs(b, b->runs, t));
    mcgb_ctx *c = b->engine.get();
    b->t_mean.clear();
    b->t_sd.clear();
    size_t k = 0;
    for (auto &r : b->runs) {
        std::vector<std::vector<double>> m, s;
        for (size_t t2 = 0; t2 < r.def->tallies.size(); t2++, k++) {
            m.push_back(c->t_mean[k]);
            s.push_back(c->t_sd[k]);
        }
        b->t_mean.push_back(m);
        b->t_sd.push_back(s);
    }
    return MCGB_OK;
}

int mcgb_batch_tally(mcgb_batch *b, int problem, int tally, double *mean, double *sd, size_t cap,
                     size_t *needed)
{
    if (!b || problem < 0 || problem >= (int)b->t_mean.size() || tally < 0 ||
        tally >= (int)b->t_mean[problem].size())
        return fail(MCGB_E_NOT_FOUND, "no such tally result");
    size_t n = b->t_mean[problem][tally].size();
    if (needed) *needed = n;
    if (cap < n) return fail(MCGB_E_INVALID_ARG, "output capacity too small");
    if (mean) std::memcpy(mean, b->t_mean[problem][tally].data(), n * 8);
    if (sd) std::memcpy(sd, b->t_sd[problem][tally].data(), n * 8);
    return MCGB_OK;
}

int mcgb_batch_counters(mcgb_batch *b, mcgb_counters *out)
{
    if (!b || !out || !b->engine) return fail(MCGB_E_STATE, "batch has not run");
    *out = b->engine->counters;
    return MCGB_OK;
}

}  // extern "C"
