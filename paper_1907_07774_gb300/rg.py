"""Thin ctypes binding of the registration entry points (include/rg.h), same
names as the C ABI.  Argument marshalling only: the state, adjoint,
gradient, Hessian-vector and preconditioner computations run in the CUDA
library; loading fails loudly when it has not been built."""

from __future__ import annotations

import ctypes

import numpy as np

from . import rd as _rd

RD_FP64, RD_MIXED = _rd.RD_FP64, _rd.RD_MIXED


class rg_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nt", ctypes.c_int), ("prec", ctypes.c_int), ("beta_v", ctypes.c_double)]


_declared = False


def lib():
    """The shared library with the rg_* signatures declared."""
    global _declared
    L = _rd.lib()
    if not _declared:
        vp, st = ctypes.c_void_p, ctypes.c_int
        sig = {
            "rg_config_default": ([ctypes.POINTER(rg_config)], st),
            "rg_create": ([ctypes.POINTER(vp), ctypes.POINTER(rg_config), vp], st),
            "rg_set_images": ([vp, vp, vp, vp, vp], st),
            "rg_forward": ([vp, vp, vp, ctypes.POINTER(ctypes.c_double)], st),
            "rg_gradient": ([vp, vp, ctypes.POINTER(ctypes.c_double), vp], st),
            "rg_hessvec": ([vp, vp, vp, vp], st),
            "rg_apply_precond": ([vp, vp, vp], st),
            "rg_project": ([vp, vp, vp], st),
            "rg_last_error": ([vp], ctypes.c_char_p),
            "rg_destroy": ([vp], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _declared = True
    return L


def _vec(fields):
    """Array of three field pointers plus keep-alive objects."""
    ptrs, keep = [], []
    for f in fields:
        p, k = _rd._ptr(f)
        ptrs.append(p)
        keep.append(k)
    return (ctypes.c_void_p * 3)(*ptrs), keep


class RegContext:
    """One registration problem: grid, nt, precision, beta_v; the context
    owns its device memory and runs on the given (or current) stream."""

    def __init__(self, n, nt, prec="fp64", beta_v=1e-2, stream=None):
        import torch
        L = lib()
        cfg = rg_config()
        L.rg_config_default(ctypes.byref(cfg))
        n = (n, n, n) if np.isscalar(n) else tuple(n)
        for a in range(3):
            cfg.n[a] = int(n[a])
        cfg.nt = int(nt)
        cfg.prec = RD_MIXED if prec in ("mixed", RD_MIXED) else RD_FP64
        cfg.beta_v = float(beta_v)
        self.cfg, self.n = cfg, n
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = L.rg_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream))
        if st != _rd.RD_OK:
            raise _rd.RDError(st, "rg_create")
        self.h = h

    def _call(self, status):
        if status != _rd.RD_OK:
            raise _rd.RDError(status, lib().rg_last_error(self.h).decode())

    def _zeros3(self):
        return [np.zeros(self.n) for _ in range(3)]

    def rg_set_images(self, m_atlas, m_patient, c1, q=None):
        ma, k1 = _vec(m_atlas)
        mp, k2 = _vec(m_patient)
        c, k3 = _rd._ptr(c1)
        qq, k4 = _vec(q) if q is not None else (None, None)
        self._call(lib().rg_set_images(self.h, ma, mp, c, qq))

    def rg_forward(self, v, m1_out=None):
        vv, k1 = _vec(v)
        mo, k2 = _vec(m1_out) if m1_out is not None else (None, None)
        J = ctypes.c_double()
        self._call(lib().rg_forward(self.h, vv, mo, ctypes.byref(J)))
        return J.value

    def rg_gradient(self, v, g=None):
        g = self._zeros3() if g is None else g
        vv, k1 = _vec(v)
        gg, k2 = _vec(g)
        J = ctypes.c_double()
        self._call(lib().rg_gradient(self.h, vv, ctypes.byref(J), gg))
        return J.value, g

    def rg_hessvec(self, v, vt, hv=None):
        hv = self._zeros3() if hv is None else hv
        vv, k1 = _vec(v)
        tt, k2 = _vec(vt)
        hh, k3 = _vec(hv)
        self._call(lib().rg_hessvec(self.h, vv, tt, hh))
        return hv

    def rg_apply_precond(self, r, z=None):
        z = self._zeros3() if z is None else z
        rr, k1 = _vec(r)
        zz, k2 = _vec(z)
        self._call(lib().rg_apply_precond(self.h, rr, zz))
        return z

    def rg_project(self, w, kw=None):
        kw = self._zeros3() if kw is None else kw
        ww, k1 = _vec(w)
        kk, k2 = _vec(kw)
        self._call(lib().rg_project(self.h, ww, kk))
        return kw

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and _rd._lib is not None:
            _rd._lib.rg_destroy(h)


def context_for(prob, prec="fp64"):
    """Context with the images of a :class:`synth.RegistrationProblem`."""
    ctx = RegContext(prob.n, prob.nt, prec=prec, beta_v=prob.beta_v)
    ctx.rg_set_images(prob.m_atlas, prob.m_patient, prob.c1, prob.q)
    return ctx
