// kernels_aux.cu -- single building blocks of the transport run alone on the
// device, so that they can be compared one by one with other implementations.
#include "kernels.h"
#include "transport.cuh"

namespace mcgb {

__global__ void k_rng_states(uint64_t seed, uint64_t first_id, int64_t n, int draws, uint64_t *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t s = rng_stream(seed, first_id + (uint64_t)i);
    for (int k = 0; k < draws; k++) {
        s = rng_next(s);
        out[i * draws + k] = s;
    }
}

void launch_rng_states(uint64_t seed, uint64_t first_id, int64_t n, int draws, uint64_t *out,
                       cudaStream_t st)
{
    if (n <= 0) return;
    k_rng_states<<<(int)((n + 255) / 256), 256, 0, st>>>(seed, first_id, n, draws, out);
}

// FP64 throughput probe: each thread runs FP64_CHAINS independent fused
// multiply-add chains of `iters` steps, so with enough resident warps the FP64
// pipe, not its latency, sets the rate.  x -> a x + b with 0 < a < 1 stays
// finite and positive; the sum is stored only if negative (never), so the
// compiler cannot drop the chains.
constexpr int FP64_CHAINS = 8;

__global__ void __launch_bounds__(256) k_fp64_rate(long long iters, double a, double b,
                                                   double *sink)
{
    double x[FP64_CHAINS];
#pragma unroll
    for (int k = 0; k < FP64_CHAINS; k++) x[k] = 1e-3 * (double)threadIdx.x + (double)k;
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < FP64_CHAINS; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < FP64_CHAINS; k++) s += x[k];
    if (s < 0.0) sink[blockIdx.x] = s;
}

int fp64_rate_chains() { return FP64_CHAINS; }

void launch_fp64_rate(int grid, long long iters, double *sink, cudaStream_t st)
{
    k_fp64_rate<<<grid, 256, 0, st>>>(iters, 0.999999, 1e-6, sink);
}

__global__ void k_log(World W, int64_t n, const double *xi, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = xi[i];
    // only the xi of the generator: k 2^-53 with k in [1, 2^53]
    if (!(x > 0.0) || x > 1.0) {
        out[i] = __longlong_as_double(0x7FF8000000000000LL);
        return;
    }
    uint64_t k = (uint64_t)(x * 9007199254740992.0);
    out[i] = log_n(W, k);
}

void launch_log(const World &W, int64_t n, const double *xi, double *out, cudaStream_t st)
{
    if (n <= 0) return;
    k_log<<<(int)((n + 255) / 256), 256, 0, st>>>(W, n, xi, out);
}

__global__ void k_fpint_ops(int64_t n, const double *a, const double *b, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = a[i], y = b[i];
    out[3 * i] = sqrt_rn(x);
    out[3 * i + 1] = div_rn(x, y);
    out[3 * i + 2] = rcp_rn(y);
}

void launch_fpint_ops(int64_t n, const double *a, const double *b, double *out, cudaStream_t st)
{
    if (n <= 0) return;
    k_fpint_ops<<<(int)((n + 255) / 256), 256, 0, st>>>(n, a, b, out);
}

__global__ void k_probe(World W, int root_univ, int64_t n, const double *pos, const double *dir,
                        int *path, double *dist, int *kind)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PS p;
    p.x = pos[3 * i]; p.y = pos[3 * i + 1]; p.z = pos[3 * i + 2];
    p.u = dir[3 * i]; p.v = dir[3 * i + 1]; p.w = dir[3 * i + 2];
    set_recip(W, p);
    p.ix = p.iy = p.ucell = -1;
    p.cell = p.mat = -1;
    if (!locate_full(W, root_univ, p)) {
        for (int k = 0; k < 5; k++) path[5 * i + k] = -1;
        dist[i] = -1.0;
        kind[i] = -1;
        return;
    }
    path[5 * i] = p.cell; path[5 * i + 1] = p.ix; path[5 * i + 2] = p.iy;
    path[5 * i + 3] = p.ucell; path[5 * i + 4] = p.mat;
    int kd, which;
    dist[i] = boundary(W, p, kd, which);
    kind[i] = kd;
}

void launch_probe(const World &W, int root_univ, int64_t n, const double *pos, const double *dir,
                  int *path, double *dist, int *kind, cudaStream_t st)
{
    if (n <= 0) return;
    k_probe<<<(int)((n + 127) / 128), 128, 0, st>>>(W, root_univ, n, pos, dir, path, dist, kind);
}

__global__ void k_ce_lookup(World W, int mat, int64_t n, const double *E, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double e = E[i];
    int k = union_index(W, e);
    double sigt, nusf;
    ce_macro(W, mat, e, sigt, nusf);
    int off = W.mc_off[mat], nn = W.mc_n[mat];
    double ss = 0.0, sf = 0.0;
    for (int q = 0; q < nn; q++) {
        double a, b, c;
        ce_micro(W, W.mc_nuc[off + q], k, e, a, b, c);
        ss = ss + W.mc_dens[off + q] * b;
        sf = sf + W.mc_dens[off + q] * c;
    }
    out[4 * i] = sigt;
    out[4 * i + 1] = nusf;
    out[4 * i + 2] = ss;
    out[4 * i + 3] = sf;
}

void launch_ce_lookup(const World &W, int mat, int64_t n, const double *E, double *out,
                      cudaStream_t st)
{
    if (n <= 0) return;
    k_ce_lookup<<<(int)((n + 127) / 128), 128, 0, st>>>(W, mat, n, E, out);
}

}  // namespace mcgb
