// kernels_grad.cu -- likelihood-ratio derivatives of a detector tally by
// replay (the paper has no counterpart; this is the textbook score-function
// estimator).  dE[T]/dtheta = E[sum_e s_e D_e]: s_e is the derivative of the
// log-probability of event e and D_e the tally scored from the start of e's
// flight onward by the particle plus the full subtree tallies of the
// secondaries it banks at or after e.  The forward pass keeps only each
// particle's own detector tally; the backward kernel regenerates every history
// from its random stream (recomputation instead of stored tracks) and weighs
// each score with D_e, built from suffix sums of the own tally and of the
// children's subtree totals.
//
// Scores (weight 1) for material m, group g:
//   flight ending at a surface        dSigma_t: -d
//   flight ending in a collision      dSigma_t: 1/Sigma_t - d
//   fission count (mu = nuSigma_f/Sigma_t, frac mu > 0)
//                                     dnuSigma_f: f/Sigma_t, dSigma_t: -f mu/Sigma_t,
//                                     f = 1/frac (n = floor+1) or -1/(1-frac)
//   scatter g -> g'                   dSigma_s[g,g']: 1/Sigma_s[g,g'], dSigma_t: -1/Sigma_t
//   absorption (Sigma_a = Sigma_t - Sigma_s,tot > 0)
//                                     dSigma_t: 1/Sigma_a - 1/Sigma_t, dSigma_s[g,*]: -1/Sigma_a
// Parameters equal to 0 take no score.
// the float64 fallbacks of the integer-pipe square root and division inlined
// here: the replay loop is faster with them inline than with calls
#define MCGB_FALLBACK_INLINE
#include "kernels.h"
#include "steps.cuh"

namespace mcgb {

// subtree total of every slot: own (weighted over groups) + children's subtrees
__global__ void k_subtree(const double *own, const double *w, int G, int64_t n,
                          const double *sub_next, const int *off, const int *nfis, double *sub)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int g = 0; g < G; g++) s += w[g] * own[j * G + g];
    if (sub_next) {
        int o = off[j], k = nfis[j];
        for (int i = 0; i < k; i++) s += sub_next[o + i];
    }
    sub[j] = s;
}

void launch_subtree(const double *own, const double *w, int G, int64_t n, const double *sub_next,
                    const int *off, const int *nfis, double *sub, cudaStream_t st)
{
    if (n <= 0) return;
    k_subtree<<<(int)((n + 255) / 256), 256, 0, st>>>(own, w, G, n, sub_next, off, nfis, sub);
}

__global__ void __launch_bounds__(256) k_replay(World W, ReplayArgs a, Bank Bsrc)
{
    extern __shared__ double sg[];
    const int G = a.G, nm = a.nmat;
    const int npar = nm * G * (G + 2);
    for (int k = threadIdx.x; k < npar; k += blockDim.x) sg[k] = 0.0;
    __syncthreads();
    const ProblemDev &Pd = W.prob[0];
    RunBufs R{};
    Bank none{};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        PS p;
        if (!init_particle<false>(W, Pd, Bsrc, p, 0, j, a.gen, a.site ? a.site[j] : -1, false)) continue;
        double own_total = 0.0;
        for (int g = 0; g < G; g++) own_total += a.w[g] * a.own[j * G + g];
        double c_total = 0.0;
        int coff = 0;
        if (a.sub_next) {
            coff = a.off[j];
            for (int i = 0; i < a.nfis[j]; i++) c_total += a.sub_next[coff + i];
        }
        double own_before = 0.0, c_prefix = 0.0;
        double kt = 0.0, kc = 0.0;
        for (;;) {
            int kind, which, uk = 0;
            double d = 0.0;
            int g0 = p.g, m0 = p.mat;
            bool in_det = (p.ucell >= 0 ? p.ucell : p.cell) == a.det_cell;
            int ev = step_advance<true, false, false>(W, Pd, p, (int)j, R, 0, kind, which, uk, kt, &d);
            if (ev == EV_DEAD) break;
            double ownb = own_before;
            if (in_det) own_before = own_before + a.w[g0] * d;
            double D = (own_total - ownb) + (c_total - c_prefix);
            int go = __ldg(W.m_goff + m0) + g0;
            double sigt = __ldg(W.g_sigt + go);
            int it = m0 * G + g0;
            if (ev == EV_CROSS) {
                if (sigt != 0.0) atomicAdd(sg + it, -d * D);
                if (step_cross(W, p, kind, which) == EV_DEAD) break;
                continue;
            }
            double mfp = __ldg(W.g_mfp + go);
            atomicAdd(sg + it, (mfp - d) * D);
            int nfb = p.nfis, nf = 0;
            ev = step_collide<true, true, false>(W, Pd, p, (int)j, none, R, 0, kc, &nf);
            double nusf = __ldg(W.g_nusf + go), mufr = __ldg(W.g_mufr + go);
            if (nusf != 0.0 && mufr != 0.0) {
                double fac = nf > (int)__ldg(W.g_mufl + go) ? 1.0 / mufr : -1.0 / (1.0 - mufr);
                atomicAdd(sg + nm * G + nm * G * G + it, mfp * fac * D);
                atomicAdd(sg + it, -(__ldg(W.g_mu + go) * mfp) * fac * D);
            }
            if (a.sub_next)
                for (int i = 0; i < nf; i++) c_prefix += a.sub_next[coff + nfb + i];
            const double *sigs = W.gg_sigs + __ldg(W.m_ggoff + m0) + g0 * G;
            if (p.fate == FATE_ABSORBED) {
                double sa = sigt - __ldg(W.g_stot + go);
                if (sa > 0.0) {
                    atomicAdd(sg + it, (1.0 / sa - mfp) * D);
                    for (int h = 0; h < G; h++)
                        if (__ldg(sigs + h) != 0.0)
                            atomicAdd(sg + nm * G + it * G + h, -1.0 / sa * D);
                }
            } else {
                atomicAdd(sg + nm * G + it * G + p.g, 1.0 / __ldg(sigs + p.g) * D);
                atomicAdd(sg + it, -mfp * D);
            }
            if (ev == EV_DEAD) break;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < npar; k += blockDim.x)
        if (sg[k] != 0.0) atomicAdd(a.grad + k, sg[k]);
}

void launch_replay(const World &W, const ReplayArgs &a, int block, cudaStream_t st)
{
    if (a.n <= 0) return;
    int npar = a.nmat * a.G * (a.G + 2);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (a.n + block - 1) / block;
    int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    Bank b = a.bank ? *a.bank : Bank{};
    k_replay<<<grid, block, sizeof(double) * npar, st>>>(W, a, b);
}

}  // namespace mcgb

// ---------------------------------------------------------------------------
// Device-side counterparts of the host steps around the derivative path, so
// that callers holding their data on the device (torch tensors) need no host
// copies.

namespace mcgb {

// New multigroup tables of materials [first, first + nmat) from device arrays
// sigma_t [nmat][G], sigma_s [nmat][G][G] ([from][to]), nu_sigma_f [nmat][G]:
// one thread per (material, group) row writes the row and its derived
// constants with the same expressions the world builder evaluates on the host
// (1/Sigma_t, mu = nuSigma_f/Sigma_t, floor and fraction, Sigma_s,tot/Sigma_t,
// the scattering cdf).  A negative value or Sigma_s,tot > Sigma_t sets *bad
// and leaves that row untouched.
__global__ void k_update_mg(World W, int first, int nmat, int G, const double *sigt,
                            const double *sigs, const double *nusf, int *bad)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nmat * G) return;
    int mi = r / G, g = r - mi * G;
    int m = first + mi;
    const double st = sigt[r], nf = nusf[r];
    const double *row = sigs + (int64_t)r * G;
    bool ok = st >= 0.0 && nf >= 0.0;
    double acc = 0.0;
    for (int h = 0; h < G; h++) {
        ok = ok && row[h] >= 0.0;
        acc = acc + row[h];
    }
    ok = ok && !(acc > st);
    if (!ok) {
        atomicOr(bad, 1);
        return;
    }
    const int go = W.m_goff[m] + g, gg = W.m_ggoff[m] + g * G;
    double *g_sigt = const_cast<double *>(W.g_sigt), *g_nusf = const_cast<double *>(W.g_nusf);
    double *g_stot = const_cast<double *>(W.g_stot), *g_mfp = const_cast<double *>(W.g_mfp);
    double *g_mu = const_cast<double *>(W.g_mu), *g_mufl = const_cast<double *>(W.g_mufl);
    double *g_mufr = const_cast<double *>(W.g_mufr), *g_ps = const_cast<double *>(W.g_ps);
    double *gg_sigs = const_cast<double *>(W.gg_sigs), *gg_scdf = const_cast<double *>(W.gg_scdf);
    g_sigt[go] = st;
    g_nusf[go] = nf;
    g_stot[go] = acc;
    g_mfp[go] = st > 0.0 ? 1.0 / st : MCGB_INF;
    double mu = st > 0.0 ? nf / st : 0.0;
    double fl = floor(mu);
    g_mu[go] = mu;
    g_mufl[go] = fl;
    g_mufr[go] = mu - fl;
    g_ps[go] = st > 0.0 ? acc / st : 0.0;
    double run = 0.0;
    for (int h = 0; h < G; h++) {
        gg_sigs[gg + h] = row[h];
        run = run + row[h];
        gg_scdf[gg + h] = acc > 0.0 ? (h == G - 1 ? 1.0 : run / acc) : 1.0;
    }
}

// material fissile flags after an update: any nuSigma_f > 0
__global__ void k_update_fissile(World W, int first, int nmat, int G)
{
    int mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= nmat) return;
    int m = first + mi;
    int fis = 0;
    for (int g = 0; g < G; g++) fis |= W.g_nusf[W.m_goff[m] + g] > 0.0;
    const_cast<int *>(W.m_fissile)[m] = fis;
}

void launch_update_mg(const World &W, int first, int nmat, int G, const double *sigt,
                      const double *sigs, const double *nusf, int *bad, cudaStream_t st)
{
    int rows = nmat * G;
    k_update_mg<<<(rows + 127) / 128, 128, 0, st>>>(W, first, nmat, G, sigt, sigs, nusf, bad);
    k_update_fissile<<<(nmat + 127) / 128, 128, 0, st>>>(W, first, nmat, G);
}

// out[q] (+)= sum_j own[j G + q]: one block per group, a fixed reduction order
__global__ void k_own_sum(const double *own, int64_t n, int G, int accumulate, double *out)
{
    __shared__ double part[256];
    int q = blockIdx.x;
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s += own[j * G + q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = accumulate ? out[q] + part[0] : part[0];
}

void launch_own_sum(const double *own, int64_t n, int G, int accumulate, double *out,
                    cudaStream_t st)
{
    k_own_sum<<<G, 256, 0, st>>>(own, n, G, accumulate, out);
}

// dst[k] = src[k] / N for k < n
__global__ void k_scale(const double *src, int64_t n, double N, double *dst)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = src[k] / N;
}

void launch_scale(const double *src, int64_t n, double N, double *dst, cudaStream_t st)
{
    if (n > 0) k_scale<<<(int)((n + 255) / 256), 256, 0, st>>>(src, n, N, dst);
}

}  // namespace mcgb
