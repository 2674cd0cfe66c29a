// kernels_cycle.cu -- end-of-cycle work: put the fission bank in (parent,
// child) order, resample the next cycle's sources, reduce k estimators,
// counters and tallies.
//
// Bank order without a general sort: every history counts the sites it banks
// (nfis), so an exclusive scan of those counts gives each parent's first
// position; site b goes to off[parent] + child.  The order is the unique
// (parent, child) order whatever order the sites were appended in.
#include <mutex>
#include <string>

#include "kernels.h"
#include "transport.cuh"

namespace mcgb {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

int64_t scan_scratch_ints(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// Exclusive block scan of one value per thread; returns the block total in *tot.
__device__ __forceinline__ int block_exclusive_scan(int v, int *tot)
{
    __shared__ int warp_sums[SCAN_BLOCK / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    int before = wid ? warp_sums[wid - 1] : 0;
    *tot = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tile(const int *in, int *out, int64_t n,
                                                          int *tile_sums)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int ex = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums in place; grand total to *total.
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(int *tile_sums, int ntiles, int *total)
{
    int carry = 0;
    for (int b = 0; b < ntiles; b += SCAN_BLOCK) {
        int i = b + threadIdx.x;
        int v = i < ntiles ? tile_sums[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, &tot);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int *out, int64_t n, const int *tile_sums)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / SCAN_TILE];
}

void scan_exclusive(const int *in, int *out, int64_t n, int *total, int *scratch, cudaStream_t st)
{
    int ntiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (ntiles == 0) {
        cudaMemsetAsync(total, 0, sizeof(int), st);
        return;
    }
    k_scan_tile<<<ntiles, SCAN_BLOCK, 0, st>>>(in, out, n, scratch);
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(scratch, ntiles, total);
    if (ntiles > 1) k_scan_add<<<(int)((n + 255) / 256), 256, 0, st>>>(out, n, scratch);
}

// perm[off[parent] + child] = b for every appended site b < M.  After a bank
// overflow (M > capacity, reported to the host) only stored sites are placed.
__global__ void k_perm(const int *parent, const int *child, const int *off, const int *M, int *perm,
                       int64_t cap)
{
    int64_t m = *M < cap ? (int64_t)*M : cap;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t dst = (int64_t)off[parent[b]] + child[b];
        if (dst < cap) perm[dst] = (int)b;
    }
}

void launch_perm(const Bank &B, const int *off, const int *M, int *perm, int grid, cudaStream_t st)
{
    k_perm<<<grid, 256, 0, st>>>(B.parent, B.child, off, M, perm, B.cap);
}

// Systematic resampling of M sorted sites to N sources:
// source j <- site floor((j + xi) M / N) (clamped to M - 1).
__global__ void k_resample(const int *perm, const int *Mp, int64_t N, double xi, int *src_idx,
                           int *err, int64_t cap)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int64_t M = *Mp;
    if (M > cap) {   // overflow: reported to the host, keep indices in bounds
        atomicOr(err, ERR_BANK_OVERFLOW);
        M = cap;
    }
    if (M <= 0) {   // empty bank: the host reports it and stops
        src_idx[j] = 0;
        return;
    }
    src_idx[j] = perm[site_index_of(j, xi, M, N)];
}

void launch_resample(const int *perm, const int *M, int64_t N, double xi, int *src_idx, int *err,
                     int64_t cap, cudaStream_t st)
{
    k_resample<<<(int)((N + 255) / 256), 256, 0, st>>>(perm, M, N, xi, src_idx, err, cap);
}

// Sums of per-history k estimators and event counters over the generation's slots.
__global__ void k_reduce_gen(Particles P, int64_t total, const int *total_dev, double *kout,
                             unsigned long long *cnt, const int *cyc_dev)
{
    int64_t n = total_dev ? (int64_t)*total_dev : total;
    if (cyc_dev) kout += 2 * *cyc_dev;
    double kt = 0.0, kc = 0.0;
    unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        kt += P.kt[i];
        kc += P.kc[i];
        c[0] += P.ncoll[i];
        c[1] += P.ncross[i];
        int f = P.fate[i];
        c[2] += f == FATE_LEAKED;
        c[3] += f == FATE_LOST;
        c[4] += f == FATE_CAPPED;
        c[5] += f == FATE_TIME;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kt += __shfl_down_sync(0xffffffffu, kt, o);
        kc += __shfl_down_sync(0xffffffffu, kc, o);
#pragma unroll
        for (int q = 0; q < 6; q++) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
    }
    // the block's warps combine in shared memory: one set of atomics per block
    __shared__ double wk[2][8];
    __shared__ unsigned long long wc[6][8];
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        wk[0][warp] = kt;
        wk[1][warp] = kc;
#pragma unroll
        for (int q = 0; q < 6; q++) wc[q][warp] = c[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; w++) {
            kt += wk[0][w];
            kc += wk[1][w];
#pragma unroll
            for (int q = 0; q < 6; q++) c[q] += wc[q][w];
        }
        atomicAdd(kout, kt);
        atomicAdd(kout + 1, kc);
#pragma unroll
        for (int q = 0; q < 6; q++)
            if (c[q]) atomicAdd(cnt + q, c[q]);
    }
}

void launch_reduce_gen(const Particles &P, int64_t total, const int *total_dev, double *kout,
                       unsigned long long *cnt, cudaStream_t st, const int *cyc_dev)
{
    k_reduce_gen<<<608, 256, 0, st>>>(P, total, total_dev, kout, cnt, cyc_dev);
}

// Sum of the replicas of accumulator i, in replica order, clearing them when
// `clear`.  The loads of a batch of replicas are issued together (they do not
// wait for the previous batch's stores), so the sum is bound by memory
// throughput rather than one memory latency per replica.
constexpr int REP_BATCH = 16;

__device__ __forceinline__ double sum_replicas(double *tacc, int acc_size, int nrep, int i, bool clear)
{
    double v = 0.0;
    for (int r0 = 0; r0 < nrep; r0 += REP_BATCH) {
        double a[REP_BATCH];
#pragma unroll
        for (int q = 0; q < REP_BATCH; q++)
            a[q] = r0 + q < nrep ? __ldcg(tacc + (int64_t)(r0 + q) * acc_size + i) : 0.0;
#pragma unroll
        for (int q = 0; q < REP_BATCH; q++)
            if (r0 + q < nrep) {
                v += a[q];
                if (clear) tacc[(int64_t)(r0 + q) * acc_size + i] = 0.0;
            }
    }
    return v;
}

// Eigenvalue cycle end: batch value v = (sum of replicas) / N; keep sum and
// sum of squares over active cycles; clear the accumulators.
__global__ void k_tally_cycle(double *tacc, int acc_size, int nrep, double n, int active,
                              double *tsum, double *tsum2, const int *cyc_dev, int inactive)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= acc_size) return;
    if (cyc_dev) active = *cyc_dev >= inactive;
    double v = sum_replicas(tacc, acc_size, nrep, i, true);
    v = v / n;
    if (active) {
        tsum[i] += v;
        tsum2[i] += v * v;
    }
}

void launch_tally_cycle(double *tacc, int acc_size, int nrep, double n, int active,
                        double *tsum, double *tsum2, cudaStream_t st, const int *cyc_dev,
                        int inactive)
{
    if (acc_size <= 0) return;
    k_tally_cycle<<<(acc_size + 63) / 64, 64, 0, st>>>(tacc, acc_size, nrep, n, active, tsum,
                                                       tsum2, cyc_dev, inactive);
}

__global__ void k_resample_dev(const int *perm, const int *Mp, int64_t N, const double *xi_tab,
                               const int *cyc_dev, int *src_idx, int *err, int64_t cap)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double xi = xi_tab[*cyc_dev];
    int64_t M = *Mp;
    if (M > cap) {
        atomicOr(err, ERR_BANK_OVERFLOW);
        M = cap;
    }
    if (M <= 0) {
        src_idx[j] = 0;
        return;
    }
    src_idx[j] = perm[site_index_of(j, xi, M, N)];
}

void launch_resample_dev(const int *perm, const int *M, int64_t N, const double *xi_tab,
                         const int *cyc_dev, int *src_idx, int *err, int64_t cap, cudaStream_t st)
{
    k_resample_dev<<<(int)((N + 255) / 256), 256, 0, st>>>(perm, M, N, xi_tab, cyc_dev, src_idx,
                                                           err, cap);
}

__global__ void k_cycle_end(int *cyc_dev, const int *M, int64_t *bank_m)
{
    bank_m[*cyc_dev] = *M;
    *cyc_dev += 1;
}

void launch_cycle_end(int *cyc_dev, const int *M, int64_t *bank_m, cudaStream_t st)
{
    k_cycle_end<<<1, 1, 0, st>>>(cyc_dev, M, bank_m);
}

__global__ void k_acc_reduce(const double *tacc, int acc_size, int nrep, double *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= acc_size) return;
    out[i] = sum_replicas(const_cast<double *>(tacc), acc_size, nrep, i, false);
}

void launch_acc_reduce(const double *tacc, int acc_size, int nrep, double *out, cudaStream_t st)
{
    k_acc_reduce<<<(acc_size + 63) / 64, 64, 0, st>>>(tacc, acc_size, nrep, out);
}

// First slot of each problem in the next generation: off[base[p]] (M past the end).
__global__ void k_gen_base(const int64_t *base, int nprob, const int *off, const int *M,
                           int64_t *next)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nprob) return;
    int64_t total = base[nprob];
    next[p] = base[p] < total ? (int64_t)off[base[p]] : (int64_t)*M;
}

void launch_gen_base(const int64_t *base, int nprob, const int *off, const int *M,
                     int64_t *next_base, cudaStream_t st)
{
    k_gen_base<<<(nprob + 1 + 127) / 128, 128, 0, st>>>(base, nprob, off, M, next_base);
}

__global__ void k_copy_records(Particles P, int64_t n, int *ncoll, int *ncross, uint64_t *rng,
                               int *nfis, int *fate, int *g)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ncoll[i] = P.ncoll[i];
    ncross[i] = P.ncross[i];
    rng[i] = P.s[i];
    nfis[i] = P.nfis[i];
    fate[i] = P.fate[i];
    g[i] = P.g[i];
}

void launch_copy_records(const Particles &P, int64_t n, int *ncoll, int *ncross, uint64_t *rng,
                         int *nfis, int *fate, int *g, cudaStream_t st)
{
    if (n <= 0) return;
    k_copy_records<<<(int)((n + 255) / 256), 256, 0, st>>>(P, n, ncoll, ncross, rng, nfis, fate, g);
}

}  // namespace mcgb

// ---------------------------------------------------------------------------
// Allocation-free bank offsets.
//
// Some callers cannot give this library device memory of its own: their device
// memory is owned by another allocator (a framework's caching allocator that
// has reserved the GPU), or they must not allocate once they are running
// (latency-critical loops).  This entry point does the bank-ordering scan with
// its tile sums in a fixed array compiled into the library instead of a
// buffer from cudaMalloc.  Every GPU that loads the library holds the array
// (16 KiB) until the process exits.
namespace mcgb {
int set_error(int code, const char *msg);
}

namespace {

constexpr int NOALLOC_MAX_TILES = 4096;   // n <= 4096 tiles x 4096 counts = 16,777,216

// Tile sums of the allocation-free scan.  Host code must not pass this name to a
// kernel (on the host it is only a stand-in); it passes the device address
// found once per device with cudaGetSymbolAddress.
static __device__ __align__(256) int g_noalloc_tiles[NOALLOC_MAX_TILES];

std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
int *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

}  // namespace

extern "C" int mcgb_bank_offsets_noalloc(const int32_t *n_fis, int64_t n, int32_t *first,
                                         int32_t *total, void *cuda_stream)
{
    using namespace mcgb;
    if (n < 0 || (n > 0 && (!n_fis || !first)) || !total)
        return set_error(-1, "mcgb_bank_offsets_noalloc: null pointer or negative n");
    if (n > (int64_t)NOALLOC_MAX_TILES * SCAN_TILE)
        return set_error(-1, "mcgb_bank_offsets_noalloc: n exceeds the maximum of 16777216 counts "
                             "(4096 tiles of 4096)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(-3, "mcgb_bank_offsets_noalloc: no usable current device");
    int *tiles = nullptr;
    {
        // first call on this device (with it current): look up the array's device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_noalloc_ptr[dev], g_noalloc_tiles);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                return set_error(-3, (std::string("mcgb_bank_offsets_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e)).c_str());
            }
        }
        tiles = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int ntiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (ntiles == 0) {
        e = cudaMemsetAsync(total, 0, sizeof(int32_t), st);
    } else {
        // every tile sum that is read is written first by k_scan_tile: nothing needs clearing
        k_scan_tile<<<ntiles, SCAN_BLOCK, 0, st>>>(n_fis, first, n, tiles);
        k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(tiles, ntiles, total);
        if (ntiles > 1) k_scan_add<<<(int)((n + 255) / 256), 256, 0, st>>>(first, n, tiles);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_error(-3, (std::string("mcgb_bank_offsets_noalloc: ") + cudaGetErrorString(e)).c_str());
    return 0;
}

// ---------------------------------------------------------------------------
// Sharded power iteration: one rank's share of the per-cycle exchange.

namespace mcgb {

// The rank's sites in (parent, child) order as records: out[k] = site perm[k]
// of B, its parent made global (j0 + local index).
__global__ void k_pack_sites(Bank B, const int *perm, int64_t M, int64_t j0, ShardSite *out)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    int b = perm[k];
    ShardSite s;
    s.x = B.x[b];
    s.y = B.y[b];
    s.z = B.z[b];
    s.t = B.t[b];
    s.cell = B.cell[b];
    s.ix = B.ix[b];
    s.iy = B.iy[b];
    s.ucell = B.ucell[b];
    s.mat = B.mat[b];
    s.child = B.child[b];
    s.parent = j0 + B.parent[b];
    out[k] = s;
}

void launch_pack_sites(const Bank &B, const int *perm, int64_t M, int64_t j0, ShardSite *out,
                       cudaStream_t st)
{
    if (M > 0) k_pack_sites<<<(int)((M + 255) / 256), 256, 0, st>>>(B, perm, M, j0, out);
}

// Sources j0 .. j0+n-1 of the next cycle from the global ordered bank of M
// sites: systematic resampling with the cycle's draw (site_index_of, exactly as
// a single device resamples), written as the birth bank Bs in local order.
__global__ void k_unpack_sources(const ShardSite *bank, int64_t M, int64_t N, int64_t j0, int64_t n,
                                 double xi, Bank Bs)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const ShardSite &s = bank[site_index_of(j0 + k, xi, M, N)];
    Bs.x[k] = s.x;
    Bs.y[k] = s.y;
    Bs.z[k] = s.z;
    Bs.t[k] = s.t;
    Bs.cell[k] = s.cell;
    Bs.ix[k] = s.ix;
    Bs.iy[k] = s.iy;
    Bs.ucell[k] = s.ucell;
    Bs.mat[k] = s.mat;
}

void launch_unpack_sources(const ShardSite *bank, int64_t M, int64_t N, int64_t j0, int64_t n,
                           double xi, const Bank &Bs, cudaStream_t st)
{
    if (n > 0 && M > 0)
        k_unpack_sources<<<(int)((n + 255) / 256), 256, 0, st>>>(bank, M, N, j0, n, xi, Bs);
}

// Birth sites k = 0 .. n-1 from records in source order (a restored checkpoint:
// source j of the cycle is born at site j).
__global__ void k_sites_to_bank(const ShardSite *in, int64_t n, Bank Bs)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const ShardSite &s = in[k];
    Bs.x[k] = s.x;
    Bs.y[k] = s.y;
    Bs.z[k] = s.z;
    Bs.t[k] = s.t;
    Bs.cell[k] = s.cell;
    Bs.ix[k] = s.ix;
    Bs.iy[k] = s.iy;
    Bs.ucell[k] = s.ucell;
    Bs.mat[k] = s.mat;
    Bs.parent[k] = (int)k;
    Bs.child[k] = 0;
    Bs.root[k] = (int)k;
    Bs.prob[k] = 0;
}

void launch_sites_to_bank(const ShardSite *in, int64_t n, const Bank &Bs, cudaStream_t st)
{
    if (n > 0) k_sites_to_bank<<<(int)((n + 255) / 256), 256, 0, st>>>(in, n, Bs);
}

// Statistics of one cycle from the all-rank sums [k_tl, k_c, tally...]: the k
// sums go to kout[2 cyc ..]; in an active cycle each tally batch value
// v = sum / N is added to tsum and v^2 to tsum2 (as k_tally_cycle does).
__global__ void k_shard_stats(const double *sums, int acc_size, double N, int cyc, int active,
                              double *kout, double *tsum, double *tsum2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2) kout[2 * cyc + i] = sums[i];
    if (i >= acc_size || !active) return;
    double v = sums[2 + i] / N;
    tsum[i] += v;
    tsum2[i] += v * v;
}

void launch_shard_stats(const double *sums, int acc_size, double N, int cyc, int active,
                        double *kout, double *tsum, double *tsum2, cudaStream_t st)
{
    int n = acc_size > 2 ? acc_size : 2;
    k_shard_stats<<<(n + 255) / 256, 256, 0, st>>>(sums, acc_size, N, cyc, active, kout, tsum, tsum2);
}

}  // namespace mcgb
