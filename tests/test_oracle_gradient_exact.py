"""Exact pin of the likelihood-ratio derivatives: infinite medium, fixed source.

For one material filling a reflective cube with a uniform source of spectrum q,
the flux per source neutron is phi = B^-1 q, B = diag Sigma_t - Sigma_s^T -
chi nuSigma_f^T.  With T = w . phi:
  dT/dSigma_t[g]     = -(w B^-1)_g phi_g
  dT/dSigma_s[g,g']  = +(w B^-1)_g' phi_g
  dT/dnuSigma_f[g]   = +(w B^-1 chi) phi_g
Every score type of the estimator (flights ending at reflective surfaces and in
collisions, scattering, absorption, fission counts with secondary subtrees)
contributes, so a wrong term in any of them moves the estimate off these values.
"""
import numpy as np

import workloads as W
from oracle import Oracle


def material():
    rng = np.random.default_rng(42)
    return W.mg_material(rng, 4, fissile=True, kinf=0.6, sigt=(0.5, 1.5), ratio=(0.4, 0.9))


def exact(mat, q, w):
    B = np.diag(mat["sigma_t"]) - mat["sigma_s"].T - np.outer(mat["chi"], mat["nu_sigma_f"])
    phi = np.linalg.solve(B, q)
    adj = np.linalg.solve(B.T, w)          # w B^-1
    d_st = -adj * phi
    d_ss = np.outer(phi, adj)              # [g, g'] = adj[g'] phi[g]
    d_nf = (adj @ mat["chi"]) * phi
    return phi, d_st, d_ss, d_nf


def test_lr_derivatives_match_infinite_medium_closed_form(orc):
    mat = material()
    G = 4
    q = np.array([0.6, 0.25, 0.1, 0.05])
    w = np.array([1.0, 0.5, 2.0, 1.5])
    pb = W.infinite_medium_fixed(mat, q, half=0.4)
    phi, d_st, d_ss, d_nf = exact(mat, q, w)
    runs = []
    for k in range(10):
        g = Oracle(pb).grad(n=30000, seed=500 + k, cell=0, weights=w)
        runs.append(np.concatenate([g["tally"], g["sigma_t"][0], g["sigma_s"][0].ravel(),
                                    g["nu_sigma_f"][0]]))
    runs = np.array(runs)
    est, sd = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    ref = np.concatenate([phi, d_st, d_ss.ravel(), d_nf])
    live = np.concatenate([np.ones(G, bool), mat["sigma_t"] > 0, mat["sigma_s"].ravel() > 0,
                           mat["nu_sigma_f"] > 0])
    z = (est - ref) / np.where(sd > 0, sd, 1.0)
    assert np.all(np.abs(z[live]) < 5), list(zip(np.round(ref, 4), np.round(est, 4), np.round(z, 2)))
    # zero-valued parameters take no score
    assert np.all(est[~live] == 0.0)
