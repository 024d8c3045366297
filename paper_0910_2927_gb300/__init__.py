"""sign(H_W(mu)) b on GB300: restarted LR-deflated multishift FOM (Bloch et al., Lattice 2009).

Python layer over the C ABI of ``include/sgn.h``.  It only marshals
arguments: every step of the method runs in the CUDA kernels of libsgn.so.
PyTorch provides device memory (through its caching allocator) and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import (APPLY_ADJOINT, APPLY_HOST_BUFFERS, FORM_A, FORM_A2, HW_ADJOINT, HW_FLOAT_FLOAT, HW_PACKED,
                   LINKS_BF16, LINKS_FP16, LINKS_FP32, METHOD_FOM, METHOD_GMRES, PREC_FP64, PREC_MIXED, Report,
                   SignError, check, lib)

__all__ = ["SignContext", "kenney_laub", "SignError", "PREC_FP64", "PREC_MIXED", "LINKS_FP32", "LINKS_BF16",
           "LINKS_FP16", "HW_ADJOINT", "HW_PACKED", "HW_FLOAT_FLOAT", "FORM_A2", "FORM_A", "METHOD_FOM",
           "METHOD_GMRES", "sign_apply", "SignApply"]


def kenney_laub(s: int, c: float = 1.0):
    """Shifts and weights of eq. (6.2) with the scale c folded in (sgn_kenney_laub)."""
    sig = np.empty(s)
    om = np.empty(s)
    check(lib().sgn_kenney_laub(int(s), float(c), sig.ctypes.data, om.ctypes.data))
    return sig, om


def _torch():
    import torch
    return torch


class SignContext:
    """One lattice, one operator H_W(mu), one GPU.  Wraps an ``sgn_ctx``."""

    def __init__(self, dims, mu=0.0, mass=-1.6, antiperiodic=(0, 0, 0, 1), device=None, stream=None,
                 torch_allocator=True):
        torch = _torch()
        self.dims = tuple(int(d) for d in dims)
        self.vol = int(np.prod(self.dims))
        self.n = 12 * self.vol
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if torch_allocator:
            dev = self.device.index

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, self._stream)
                except Exception:
                    return None

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = _abi.ALLOC_FN(_alloc)
            self._free_cb = _abi.FREE_FN(_free)
        else:
            self._alloc_cb = _abi.ALLOC_FN()
            self._free_cb = _abi.FREE_FN()
        h = C.c_void_p()
        dims_c = (C.c_int * 4)(*self.dims)
        check(lib().sgn_create(C.byref(h), dims_c, self._alloc_cb, self._free_cb, None,
                               C.c_void_p(self._stream.cuda_stream)))
        self._h = h
        self.s = 0
        self.m = 0
        self.mu = None
        self._build_args = None       # (m, extra, eig_tol) of the last sgn_build_deflation
        # SignApply: when its mu differs from the context's and deflation data are present,
        # rebuild them at the new mu (True) or refuse (False, the default)
        self.rebuild_deflation_on_mu_change = False
        self.set_mu(mu)
        self.set_kernel_mass(mass)
        self.set_boundary(antiperiodic)

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sgn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- parameters ----------------------------------------------------------
    def set_mu(self, mu, rebuild_deflation=False):
        """A new mu drops deflation data (the solves then refuse with SGN_ERR_STATE until
        they are built, set or cleared); rebuild_deflation=True rebuilds them at the new mu
        with the arguments of the last build_deflation call."""
        mu = float(mu)
        changed = mu != self.mu
        args = self._build_args if (rebuild_deflation and self.m > 0) else None
        if rebuild_deflation and self.m > 0 and args is None:
            raise ValueError("rebuild_deflation: the deflation data were set, not built; set them again instead")
        self.mu = mu
        check(lib().sgn_set_mu(self._h, self.mu))
        if changed:
            self.m = 0
            if args is not None:
                self.build_deflation(*args)

    def set_kernel_mass(self, m_w):
        m_w = float(m_w)
        if m_w != getattr(self, "mass", None):
            self.m = 0
        self.mass = m_w
        check(lib().sgn_set_kernel_mass(self._h, self.mass))

    def set_boundary(self, antiperiodic):
        ap = tuple(int(bool(a)) for a in antiperiodic)
        if ap != getattr(self, "antiperiodic", None):
            self.m = 0
        self.antiperiodic = ap
        check(lib().sgn_set_boundary(self._h, (C.c_int * 4)(*ap)))

    def set_rational(self, sigma, omega):
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        check(lib().sgn_set_rational(self._h, sig.size, sig.ctypes.data, om.ctypes.data))
        self.s = sig.size

    def set_restart(self, k=40, tol=1e-10, max_cycles=1000, project_each_cycle=True):
        self.k = int(k)
        check(lib().sgn_set_restart(self._h, int(k), float(tol), int(max_cycles), int(bool(project_each_cycle))))

    def set_precision(self, precision=PREC_FP64, target_rel_err=1e-8, link_storage=LINKS_FP32):
        check(lib().sgn_set_precision(self._h, int(precision), float(target_rel_err), int(link_storage)))

    def set_formulation(self, form=FORM_A2):
        """FORM_A2: s systems in K(A^2) (eq. 6.2 as written); FORM_A: 2s systems in K(A)."""
        check(lib().sgn_set_formulation(self._h, int(form)))

    def set_method(self, method=METHOD_FOM):
        """METHOD_FOM: FOM-LR (Algorithm 1); METHOD_GMRES: GMRES-LR (restarted multishift GMRES)."""
        check(lib().sgn_set_method(self._h, int(method)))

    def set_refinement(self, k_refine=0, max_batch=0):
        """Mixed form: restart length and batch size of the correction solves (0: defaults)."""
        check(lib().sgn_set_refinement(self._h, int(k_refine), int(max_batch)))

    # -- data ----------------------------------------------------------------
    def _as_c128(self, a):
        torch = _torch()
        if isinstance(a, torch.Tensor):
            t = a.to(torch.complex128).contiguous()
            return t, int(t.data_ptr()), int(t.is_cuda)
        arr = np.ascontiguousarray(a, dtype=np.complex128)
        return arr, arr.ctypes.data, 0

    def load_gauge(self, links):
        """links: (V, 4, 3, 3) complex128, torch (CPU or CUDA) or numpy."""
        keep, ptr, on_dev = self._as_c128(links)
        size = keep.numel() if hasattr(keep, "numel") else keep.size
        if size != self.vol * 36:
            raise ValueError(f"links must hold V*36 = {self.vol * 36} complex entries, got {size}")
        check(lib().sgn_load_gauge(self._h, C.c_void_p(ptr), on_dev))
        self.m = 0

    def set_deflation(self, R, L, lam, extra=None):
        """R, L: (n, m) right / left eigenvectors with L^dag R = I; lam: (m,) eigenvalues.
        extra = (Rx, Lx, lamx): the next eigenpairs (not deflated; used by the mu-derivative)."""
        torch = _torch()
        if R is None or (hasattr(R, "shape") and R.shape[1] == 0):
            check(lib().sgn_set_deflation(self._h, 0, None, None, None, 0))
            self.m = 0
            return
        self._set_pairs(lib().sgn_set_deflation, R, L, lam)
        self.m = R.shape[1]
        self._build_args = None
        if extra is not None:
            self._set_pairs(lib().sgn_set_deflation_extra, *extra)

    def _set_pairs(self, fn, R, L, lam):
        torch = _torch()
        m = R.shape[1]
        if isinstance(R, torch.Tensor):
            Rt = R.transpose(0, 1).to(torch.complex128).contiguous()
            Lt = L.transpose(0, 1).to(torch.complex128).contiguous()
            lt = torch.as_tensor(lam).to(device=Rt.device, dtype=torch.complex128).contiguous()
            ptrs = (Rt.data_ptr(), Lt.data_ptr(), lt.data_ptr())
            on_dev = int(Rt.is_cuda)
            if on_dev != int(lt.is_cuda):
                raise ValueError("R, L and lam must live on the same device")
            keep = (Rt, Lt, lt)
        else:
            Rt = np.ascontiguousarray(np.asarray(R).T, dtype=np.complex128)
            Lt = np.ascontiguousarray(np.asarray(L).T, dtype=np.complex128)
            lt = np.ascontiguousarray(lam, dtype=np.complex128)
            ptrs = (Rt.ctypes.data, Lt.ctypes.data, lt.ctypes.data)
            on_dev = 0
            keep = (Rt, Lt, lt)
        check(fn(self._h, int(m), C.c_void_p(ptrs[0]), C.c_void_p(ptrs[1]), C.c_void_p(ptrs[2]), on_dev))
        del keep

    def build_deflation(self, m, extra=4, eig_tol=1e-10):
        lam = np.empty(m + extra, dtype=np.complex128)
        check(lib().sgn_build_deflation(self._h, int(m), int(extra), float(eig_tol), lam.ctypes.data))
        self.m = m
        self._build_args = (int(m), int(extra), float(eig_tol))
        return lam

    def get_deflation(self):
        mm = C.c_int()
        check(lib().sgn_get_deflation(self._h, C.byref(mm), None, None, None))
        m = mm.value
        if m == 0:
            return None, None, np.zeros(0, dtype=np.complex128)
        R = np.empty((m, self.n), dtype=np.complex128)
        L = np.empty((m, self.n), dtype=np.complex128)
        lam = np.empty(m, dtype=np.complex128)
        check(lib().sgn_get_deflation(self._h, C.byref(mm), R.ctypes.data, L.ctypes.data, lam.ctypes.data))
        return R.T, L.T, lam

    # -- application ----------------------------------------------------------
    def apply(self, b, adjoint=False, shifts=False):
        """x = sign(H_W(+-mu)) b for b of shape (nrhs, n) or (n,).

        CUDA tensors run in place on the device; numpy arrays use the host-buffer
        mode of the ABI (copies inside the call).  Returns (x, report) or, with
        shifts=True (device only), (x, x_shift, report) with x_shift of shape
        (s, nrhs, n)."""
        torch = _torch()
        flags = APPLY_ADJOINT if adjoint else 0
        rep = Report()
        if isinstance(b, torch.Tensor) and b.is_cuda:
            squeeze = b.dim() == 1
            bb = b.reshape(-1, self.n).to(torch.complex128).contiguous()
            nrhs = bb.shape[0]
            x = torch.empty_like(bb)
            if shifts:
                xs = torch.empty((self.s, nrhs, self.n), dtype=torch.complex128, device=bb.device)
                code = lib().sgn_apply_shifts(self._h, C.c_void_p(bb.data_ptr()), C.c_void_p(x.data_ptr()),
                                              C.c_void_p(xs.data_ptr()), nrhs, flags, C.byref(rep))
            else:
                code = lib().sgn_apply(self._h, C.c_void_p(bb.data_ptr()), C.c_void_p(x.data_ptr()), nrhs, flags,
                                       C.byref(rep))
            if code not in (0, 3):
                check(code)
            out = x.reshape(-1) if squeeze else x
            if shifts:
                return out, xs, rep.as_dict()
            return out, rep.as_dict()
        if shifts:
            raise ValueError("per-shift iterates need CUDA tensors")
        arr = np.ascontiguousarray(b, dtype=np.complex128)
        squeeze = arr.ndim == 1
        arr2 = arr.reshape(-1, self.n)
        x = np.empty_like(arr2)
        code = lib().sgn_apply(self._h, C.c_void_p(arr2.ctypes.data), C.c_void_p(x.ctypes.data), arr2.shape[0],
                               flags | APPLY_HOST_BUFFERS, C.byref(rep))
        if code not in (0, 3):
            check(code)
        return (x.reshape(-1) if squeeze else x), rep.as_dict()

    def hessenberg(self, col=0, k=None):
        """H_k of the last restart cycle of the last FP64-form solve, column col: ((k+1), k)
        complex128 array, and the Arnoldi steps that cycle took (sgn_get_hessenberg)."""
        kk = C.c_int(0)
        k = getattr(self, "k", 40) if k is None else int(k)
        H = np.empty((k + 1, k), dtype=np.complex128)
        check(lib().sgn_get_hessenberg(self._h, int(col), H.ctypes.data, C.byref(kk)))
        return H, kk.value

    def inner_products(self, V, w):
        """<V_j, w_c> for J CUDA fields V (J, n) and nrhs CUDA fields w (nrhs, n): shape (nrhs, J)."""
        torch = _torch()
        Vc = V.reshape(-1, self.n).to(torch.complex128).contiguous()
        wc = w.reshape(-1, self.n).to(torch.complex128).contiguous()
        out = np.empty((wc.shape[0], Vc.shape[0]), dtype=np.complex128)
        check(lib().sgn_inner_products(self._h, C.c_void_p(Vc.data_ptr()), Vc.shape[0], C.c_void_p(wc.data_ptr()),
                                       wc.shape[0], out.ctypes.data))
        return out

    def hw(self, psi, precision=PREC_FP64, adjoint=False, packed=False, float_float=False):
        """H_W(mu) psi (or H_W(-mu) psi) for CUDA fields of shape (nrhs, n) or (n,);
        packed=True: psi is (and the result stays) in the packed layout of `pack`;
        float_float=True (FP64 only): float-float arithmetic on the FP32 units."""
        torch = _torch()
        dt = torch.complex128 if precision == PREC_FP64 else torch.complex64
        x = psi.to(dt).contiguous()
        out = torch.empty_like(x)
        nrhs = x.numel() // self.n
        flags = ((HW_ADJOINT if adjoint else 0) | (HW_PACKED if packed else 0) |
                 (HW_FLOAT_FLOAT if float_float else 0))
        check(lib().sgn_hw_apply(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), nrhs,
                                 int(precision), flags))
        return out

    def overlap(self, b):
        """D_ov b = b + gamma5 sign(H_W(mu)) b for CUDA fields of shape (nrhs, n) or (n,)."""
        torch = _torch()
        x = b.to(torch.complex128).contiguous()
        out = torch.empty_like(x)
        check(lib().sgn_overlap_apply(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                      x.numel() // self.n))
        return out

    def overlap_solve(self, b, tol=1e-8, k=30, max_restarts=50):
        """x = D_ov^{-1} b by restarted GMRES; returns (x, applications of D_ov, relative residual)."""
        torch = _torch()
        x = b.to(torch.complex128).contiguous()
        out = torch.empty_like(x)
        its, rr = C.c_int(0), C.c_double(0)
        check(lib().sgn_overlap_solve(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                      x.numel() // self.n, float(tol), int(k), int(max_restarts), C.byref(its),
                                      C.byref(rr)))
        return out, its.value, rr.value

    def apply_direct(self, b, k, adjoint=False):
        """Direct projection of eq. (6.3): x_P + ||r|| V_k sign(H_k) e_1 with k Arnoldi steps on A
        (no rational function, no restarts).  Returns (x, Krylov dimension used)."""
        torch = _torch()
        x = b.to(torch.complex128).contiguous()
        out = torch.empty_like(x)
        ku = C.c_int(0)
        check(lib().sgn_apply_direct(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                     x.numel() // self.n, int(k), APPLY_ADJOINT if adjoint else 0, C.byref(ku)))
        return out, ku.value

    def _layout(self, fn, psi, precision):
        torch = _torch()
        dt = torch.complex128 if precision == PREC_FP64 else torch.complex64
        x = psi.to(dt).contiguous()
        out = torch.empty_like(x)
        check(fn(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.numel() // self.n,
                 int(precision)))
        return out

    def pack(self, psi, precision=PREC_FP64):
        """Natural [site][spin][colour] fields -> the library's packed layout."""
        return self._layout(lib().sgn_pack_fields, psi, precision)

    def unpack(self, psi, precision=PREC_FP64):
        """Packed fields -> natural [site][spin][colour] order."""
        return self._layout(lib().sgn_unpack_fields, psi, precision)


def sign_apply(ctx: SignContext, b, adjoint=False):
    """x = sign(H_W(mu)) b through an existing context."""
    return ctx.apply(b, adjoint=adjoint)[0]


def __getattr__(name):
    if name == "SignApply":
        from .autograd import SignApply
        return SignApply
    raise AttributeError(name)
