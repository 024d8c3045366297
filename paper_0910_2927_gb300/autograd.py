"""torch.autograd.Function for x = sign(H_W(mu)) b through the C ABI.

Backward:
  grad_b  = sign(H_W(mu))^dag grad_x, one adjoint solve (SGN_APPLY_ADJOINT: the
            same kernels at -mu with L and R exchanged);
  grad_mu = Re <grad_x, dx/dmu>, from sgn_grad_mu (per-shift forward iterates
            and per-shift adjoint iterates, recomputed in the backward pass; with
            deflation also the motion of the deflated eigenpairs, through
            complex-shift multishift solves for the reduced resolvents).  The
            deflation data must be the eigenpairs at the forward's mu.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._abi import APPLY_ADJOINT, check, lib


def _use_mu(sctx, mu_v):
    """Put the context at mu_v.  Deflation data belong to one operator (eq. (4.1)), so a
    context that holds them moves to another mu only when it was told to rebuild them
    (sctx.rebuild_deflation_on_mu_change); otherwise the call refuses instead of
    silently solving undeflated."""
    if sctx.mu == mu_v:
        return
    if sctx.m > 0 and not sctx.rebuild_deflation_on_mu_change:
        raise ValueError(f"SignApply: mu = {mu_v} differs from the context's mu = {sctx.mu}, whose deflation "
                         "data would be lost; set sctx.rebuild_deflation_on_mu_change = True to rebuild them "
                         "at the new mu, or move the context with sctx.set_mu first")
    sctx.set_mu(mu_v, rebuild_deflation=sctx.m > 0)


class SignApply(torch.autograd.Function):
    """x = SignApply.apply(b, mu, ctx): b (nrhs, n) or (n,) complex128 CUDA, mu a real 0-d tensor.

    When mu differs from the context's mu, the context moves to it: freely without
    deflation data; with deflation data only if ctx.rebuild_deflation_on_mu_change is
    set (the data are then rebuilt at the new mu), else ValueError."""

    @staticmethod
    def forward(fctx, b, mu, sctx):
        mu_v = float(mu)
        _use_mu(sctx, mu_v)
        x, _ = sctx.apply(b)
        fctx.sctx = sctx
        fctx.mu = mu_v
        fctx.save_for_backward(b)
        return x

    @staticmethod
    def backward(fctx, gx):
        (b,) = fctx.saved_tensors
        sctx = fctx.sctx
        _use_mu(sctx, fctx.mu)
        gb = gmu = None
        g = gx.to(torch.complex128).contiguous()
        if fctx.needs_input_grad[0]:
            gb, _ = sctx.apply(g, adjoint=True)
        if fctx.needs_input_grad[1]:
            bb = b.reshape(-1, sctx.n).to(torch.complex128).contiguous()
            gg = g.reshape(-1, sctx.n).contiguous()
            nrhs = bb.shape[0]
            out = np.zeros(nrhs)
            check(lib().sgn_grad_mu(sctx._h, C.c_void_p(bb.data_ptr()), C.c_void_p(gg.data_ptr()), nrhs,
                                    out.ctypes.data))
            gmu = torch.tensor(float(out.sum()), dtype=torch.float64)
        return gb, gmu, None


def dhw_dmu(sctx, psi):
    """dH_W/dmu psi for CUDA fields (sgn_dhw_dmu_apply)."""
    x = psi.to(torch.complex128).contiguous()
    out = torch.empty_like(x)
    check(lib().sgn_dhw_dmu_apply(sctx._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                  x.numel() // sctx.n))
    return out
