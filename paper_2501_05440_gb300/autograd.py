"""torch.autograd.Function over the transport library's derivative path.

Forward: a fixed-source run returns the detector cell's track-length tally per
group (per source particle).  Backward: the library's replay kernel
regenerates every history from its random stream and accumulates
likelihood-ratio scores times the downstream detector tally, contracted with
grad_output, for the multigroup cross sections Sigma_t [M, G], Sigma_s
[M, G, G] and nuSigma_f [M, G].  PyTorch holds the tensors; all transport work
runs in the CUDA kernels.  CUDA tensors go through the device-pointer calls
(no host copies of any array, in order on the current torch stream); CPU
tensors through the host-array calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context, load_problem


def _dev(t):
    return t.detach().to(torch.float64).contiguous()


class DetectorTally(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_t, sigma_s, nu_sigma_f, engine, n, seed, det_cell):
        nmat, G = sigma_t.shape
        ctx.engine, ctx.nmat, ctx.device = engine, nmat, sigma_t.device
        if sigma_t.is_cuda:
            engine.set_stream(torch.cuda.current_stream(sigma_t.device).cuda_stream)
            st, ss, nf = _dev(sigma_t), _dev(sigma_s), _dev(nu_sigma_f)
            engine.update_material_mg_dev(0, nmat, st.data_ptr(), ss.data_ptr(), nf.data_ptr())
            tally = torch.empty(G, dtype=torch.float64, device=sigma_t.device)
            engine.forward_fixed_dev(int(n), int(seed), int(det_cell), tally.data_ptr())
            ctx.keep = (st, ss, nf)   # alive until the stream has read them
            return tally
        st = sigma_t.detach().to(torch.float64).numpy()
        ss = sigma_s.detach().to(torch.float64).numpy()
        nf = nu_sigma_f.detach().to(torch.float64).numpy()
        for m in range(nmat):
            engine.update_material_mg(m, st[m], ss[m].ravel(), nf[m])
        return torch.as_tensor(engine.forward_fixed(int(n), int(seed), int(det_cell)),
                               dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        nm = ctx.nmat
        if grad_out.is_cuda:
            G = grad_out.shape[0]
            w = _dev(grad_out)
            dst = torch.empty((nm, G), dtype=torch.float64, device=ctx.device)
            dss = torch.empty((nm, G, G), dtype=torch.float64, device=ctx.device)
            dnf = torch.empty((nm, G), dtype=torch.float64, device=ctx.device)
            ctx.engine.set_stream(torch.cuda.current_stream(ctx.device).cuda_stream)
            ctx.engine.backward_fixed_dev(w.data_ptr(), dst.data_ptr(), dss.data_ptr(),
                                          dnf.data_ptr())
            return dst, dss, dnf, None, None, None, None
        w = np.ascontiguousarray(grad_out.detach().to(torch.float64).numpy())
        d = ctx.engine.backward_fixed(w, nm)

        def to(a):
            return torch.as_tensor(a, dtype=torch.float64)

        return to(d["sigma_t"]), to(d["sigma_s"]), to(d["nu_sigma_f"]), None, None, None, None


def detector_tally(problem, sigma_t, sigma_s, nu_sigma_f, n, seed, det_cell, engine=None):
    """Detector tally [G] of a multigroup fixed-source problem as a differentiable function
    of its cross sections (tensors [M,G], [M,G,G], [M,G]); CUDA tensors stay on the
    device."""
    if engine is None:
        dev = sigma_t.device.index if sigma_t.is_cuda and sigma_t.device.index is not None else 0
        engine = load_problem(Context(device=dev), problem)
    return DetectorTally.apply(sigma_t, sigma_s, nu_sigma_f, engine, n, seed, det_cell)
