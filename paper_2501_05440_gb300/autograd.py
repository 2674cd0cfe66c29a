"""torch.autograd.Function over the transport library's derivative path.

Forward: a fixed-source run returns the detector cell's track-length tally per
group (per source particle).  Backward: the library's replay kernel
regenerates every history from its random stream and accumulates
likelihood-ratio scores times the downstream detector tally, contracted with
grad_output, for the multigroup cross sections Sigma_t [M, G], Sigma_s
[M, G, G] and nuSigma_f [M, G].  PyTorch holds the tensors; all transport work
runs in the CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context, load_problem


class DetectorTally(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, nu_sigma_f, engine, n, seed, det_cell):
        st = sigma_t.detach().to("cpu", torch.float64).numpy()
        ss = sigma_s.detach().to("cpu", torch.float64).numpy()
        nf = nu_sigma_f.detach().to("cpu", torch.float64).numpy()
        nmat = st.shape[0]
        for m in range(nmat):
            engine.update_material_mg(m, st[m], ss[m].ravel(), nf[m])
        tally = engine.forward_fixed(int(n), int(seed), int(det_cell))
        ctx.engine = engine
        ctx.nmat = nmat
        ctx.device = sigma_t.device
        return torch.as_tensor(tally, dtype=torch.float64, device=sigma_t.device)

    @staticmethod
    def backward(ctx, grad_out):
        w = np.ascontiguousarray(grad_out.detach().to("cpu", torch.float64).numpy())
        d = ctx.engine.backward_fixed(w, ctx.nmat)

        def to(a):
            return torch.as_tensor(a, dtype=torch.float64, device=ctx.device)

        return to(d["sigma_t"]), to(d["sigma_s"]), to(d["nu_sigma_f"]), None, None, None, None


def detector_tally(problem, sigma_t, sigma_s, nu_sigma_f, n, seed, det_cell, engine=None):
    """Detector tally [G] of a multigroup fixed-source problem as a differentiable function
    of its cross sections (tensors [M,G], [M,G,G], [M,G])."""
    if engine is None:
        engine = load_problem(Context(), problem)
        if torch.cuda.is_available():
            engine.set_stream(torch.cuda.current_stream().cuda_stream)
    return DetectorTally.apply(sigma_t, sigma_s, nu_sigma_f, engine, n, seed, det_cell)
