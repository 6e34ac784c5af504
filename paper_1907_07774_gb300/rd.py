"""Thin ctypes binding of ``librd`` (include/rd.h), same names as the C ABI.

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch provides the device workspace and the stream.  Loading fails loudly
when the library has not been built; there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librd.so")

RD_OK = 0
RD_ERR_NOCONV = 5
RD_FP64 = 0
RD_MIXED = 1
STATUS = {0: "RD_OK", 1: "RD_ERR_ARG", 2: "RD_ERR_SHAPE", 3: "RD_ERR_CUDA", 4: "RD_ERR_NOMEM",
          5: "RD_ERR_NOCONV", 6: "RD_ERR_NONFINITE", 7: "RD_ERR_STATE"}

_c_double_p = ctypes.POINTER(ctypes.c_double)


class rd_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nt", ctypes.c_int), ("t_end", ctypes.c_double),
                ("prec", ctypes.c_int), ("pcg_rtol", ctypes.c_double), ("pcg_maxit", ctypes.c_int),
                ("ckpt_stride", ctypes.c_int), ("k_w", ctypes.c_double * 3),
                ("rho_w", ctypes.c_double * 3), ("beta_p", ctypes.c_double), ("moving_atlas", ctypes.c_int),
                ("coupling", ctypes.c_int), ("guess_restart", ctypes.c_int)]


_lib = None


def lib():
    """Load ``librd.so`` once and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librd.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, cd, ci, st = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int
    sig = {
        "rd_config_default": ([ctypes.POINTER(rd_config)], st),
        "rd_workspace_size": ([ctypes.POINTER(rd_config), ci, ctypes.POINTER(ctypes.c_size_t)], st),
        "rd_create": ([ctypes.POINTER(vp), ctypes.POINTER(rd_config), ci, vp, ctypes.c_size_t, vp], st),
        "rd_set_tissue": ([vp, vp, vp, vp], st),
        "rd_set_basis": ([vp, vp, cd], st),
        "rd_set_data": ([vp, vp], st),
        "rd_set_anatomy_data": ([vp, vp, vp, vp], st),
        "rd_coupling_field": ([vp, vp, vp, vp], st),
        "rd_forward": ([vp, vp, cd, cd, vp, _c_double_p], st),
        "rd_adjoint": ([vp, vp], st),
        "rd_gradient": ([vp, vp, cd, cd, _c_double_p, vp], st),
        "rd_last_gradient": ([vp, vp], st),
        "rd_hessvec": ([vp, vp, cd, cd, vp, vp], st),
        "rd_apply_operator": ([vp, cd, vp, vp], st),
        "rd_apply_precond": ([vp, cd, vp, vp], st),
        "rd_set_precond_scale": ([vp, cd], st),
        "rd_last_pcg_iters": ([vp], ci),
        "rd_last_pcg_solves": ([vp], ci),
        "rd_last_graph_solves": ([vp], ci),
        "rd_batch_gradient": ([vp, ci, vp, vp, vp, vp, vp], st),
        "rd_autotune": ([vp, ci, vp, vp, ci], st),
        "rd_autotune_clear": ([], None),
        "rd_last_error": ([vp], ctypes.c_char_p),
        "rd_destroy": ([vp], None),
        "rd_apply_precond_static": ([vp, cd, vp, vp, vp], st),
        "rd_selftest_bounded_wait": ([ctypes.c_uint, ci, vp, vp, vp], st),
        "rd_probe_fma_rate": ([ci, _c_double_p], st),
        "rd_active_tiles": ([vp, vp], st),
        "rd_profile_enable": ([ci], None),
        "rd_profile_read": ([vp, vp, ci], ci),
        "rd_profile_class": ([ci], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def rd_profile_enable(on):
    lib().rd_profile_enable(1 if on else 0)


def rd_autotune_clear():
    lib().rd_autotune_clear()


def rd_profile_read():
    """{class name: (device ms, launches)} since rd_profile_enable(1)."""
    n = 16
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    k = lib().rd_profile_read(ms, cnt, n)
    return {lib().rd_profile_class(i).decode(): (ms[i], cnt[i]) for i in range(k)}


def rd_apply_precond_static(n, coef, r, z, stream=None):
    """Allocation-free preconditioner application (FP64 device tensors r,
    z); see include/rd.h.  Returns the status code."""
    import torch
    dims = (ctypes.c_int * 3)(*[int(k) for k in n])
    (a, ka), (b, kb) = _ptr(r), _ptr(z)
    st = stream if stream is not None else torch.cuda.current_stream()
    return lib().rd_apply_precond_static(dims, float(coef), a, b, ctypes.c_void_p(st.cuda_stream))


def rd_selftest_bounded_wait(polls, copy, src16, status, stream=None):
    """Self-test of the bounded device-side wait (see include/rd.h): src16 a
    16-byte CUDA tensor or None, status a one-element int32 CUDA tensor.
    Returns the status code of the launch."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    src = src16.data_ptr() if src16 is not None else None
    ptr = status.data_ptr() if status is not None else None
    return lib().rd_selftest_bounded_wait(int(polls), int(copy), src, ptr, ctypes.c_void_p(st.cuda_stream))


def rd_probe_fma_rate(prec="fp64"):
    """Measured FMA rate of the current device in TFLOP/s (see include/rd.h)."""
    v = ctypes.c_double(0.0)
    status = lib().rd_probe_fma_rate(RD_FP64 if prec == "fp64" else RD_MIXED, ctypes.byref(v))
    if status != RD_OK:
        raise RDError(status, "FMA probe failed")
    return v.value


class RDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    """Address of a contiguous FP64 numpy array or torch tensor (host or
    device); returns (pointer, keep-alive object)."""
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x, dtype=np.float64)
        return a.ctypes.data, a
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("fields must be contiguous float64 tensors")
        return x.data_ptr(), x
    raise TypeError(f"unsupported array type {type(x)}")


def _host_vec(v, n):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class Context:
    """One ``rd_ctx``: a grid, its coefficients, basis and data, and a
    workspace allocated through PyTorch on the current CUDA device."""

    def __init__(self, n, nt, np_, prec="fp64", pcg_rtol=None, pcg_maxit=200, ckpt_stride=0,
                 k_w=(1.0, 0.1, 0.0), rho_w=(1.0, 0.2, 0.0), beta_p=0.0, t_end=1.0,
                 stream=None, device=None, moving_atlas=False, coupling=False, guess_restart=0):
        import torch
        L = lib()
        cfg = rd_config()
        L.rd_config_default(ctypes.byref(cfg))
        n = (n, n, n) if np.isscalar(n) else tuple(n)
        for a in range(3):
            cfg.n[a] = int(n[a])
        cfg.nt = int(nt)
        cfg.t_end = float(t_end)
        cfg.prec = RD_MIXED if prec in ("mixed", RD_MIXED) else RD_FP64
        cfg.pcg_rtol = float(pcg_rtol if pcg_rtol is not None else (1e-6 if cfg.prec == RD_MIXED else 1e-10))
        cfg.pcg_maxit = int(pcg_maxit)
        cfg.ckpt_stride = int(ckpt_stride)
        for a in range(3):
            cfg.k_w[a] = float(k_w[a])
            cfg.rho_w[a] = float(rho_w[a])
        cfg.beta_p = float(beta_p)
        cfg.moving_atlas = 1 if moving_atlas else 0
        cfg.coupling = 1 if coupling else 0
        cfg.guess_restart = int(guess_restart)
        self.cfg = cfg
        self.n = n
        self.np = int(np_)
        nbytes = ctypes.c_size_t()
        self._check(L.rd_workspace_size(ctypes.byref(cfg), self.np, ctypes.byref(nbytes)), None)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            self._check(L.rd_create(ctypes.byref(h), ctypes.byref(cfg), self.np, ctypes.c_void_p(aligned),
                                    nbytes.value, ctypes.c_void_p(self.stream.cuda_stream)), None)
        self.h = h
        self.last_theta = None   # parameters of the trajectory the library holds

    def _remember(self, p, k_f, rho_f):
        self.last_theta = (np.array(p, dtype=np.float64).reshape(-1), float(k_f), float(rho_f))

    def _check(self, status, h):
        if status not in (RD_OK,):
            msg = lib().rd_last_error(h).decode() if h is not None and h.value else ""
            raise RDError(status, msg)

    def _call(self, status, allow_noconv=False):
        if status == RD_ERR_NOCONV and allow_noconv:
            return status
        self._check(status, self.h)
        return status

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and _lib is not None:
            _lib.rd_destroy(h)
            self.h = None

    # -- setup ------------------------------------------------------------
    def rd_set_tissue(self, m_wm, m_gm, m_csf):
        (a, ka), (b, kb), (c, kc) = _ptr(m_wm), _ptr(m_gm), _ptr(m_csf)
        self._call(lib().rd_set_tissue(self.h, a, b, c))

    def rd_set_basis(self, centers, sigma):
        cen = _host_vec(centers, 3 * self.np)
        self._call(lib().rd_set_basis(self.h, cen.ctypes.data, float(sigma)))

    def rd_set_data(self, d):
        a, k = _ptr(d)
        self._call(lib().rd_set_data(self.h, a))

    def rd_coupling_field(self, q_wm=None, q_gm=None, q_csf=None):
        """Coupling field q of the last gradient; fills the given FP64
        buffers (host arrays or CUDA tensors) or returns three new arrays."""
        if q_wm is None:
            q_wm, q_gm, q_csf = (np.zeros(self.n) for _ in range(3))
        (a, ka), (b, kb), (c, kc) = _ptr(q_wm), _ptr(q_gm), _ptr(q_csf)
        self._call(lib().rd_coupling_field(self.h, a, b, c))
        return q_wm, q_gm, q_csf

    def rd_set_precond_scale(self, scale):
        self._call(lib().rd_set_precond_scale(self.h, float(scale)))

    def rd_set_anatomy_data(self, md_wm, md_gm, md_csf):
        (a, ka), (b, kb), (c, kc) = _ptr(md_wm), _ptr(md_gm), _ptr(md_csf)
        self._call(lib().rd_set_anatomy_data(self.h, a, b, c))

    # -- solves -------------------------------------------------------------
    def rd_forward(self, p, k_f, rho_f, c1_out=None, allow_noconv=False):
        """Returns the misfit (NaN without data); writes c(1) into c1_out
        (FP64 numpy array or tensor) when given."""
        pv = _host_vec(p, self.np)
        J = ctypes.c_double(0.0)
        out = 0
        if c1_out is not None:
            out, keep = _ptr(c1_out)
        self.last_theta = None
        self._call(lib().rd_forward(self.h, pv.ctypes.data, float(k_f), float(rho_f), out, ctypes.byref(J)),
                   allow_noconv)
        self._remember(pv, k_f, rho_f)
        return J.value

    def rd_adjoint(self, alpha0_out=None, allow_noconv=False):
        out = 0
        if alpha0_out is not None:
            out, keep = _ptr(alpha0_out)
        self._call(lib().rd_adjoint(self.h, out), allow_noconv)
        g = np.zeros(self.np + 2)
        self._call(lib().rd_last_gradient(self.h, g.ctypes.data))
        return g

    def rd_gradient(self, p, k_f, rho_f, allow_noconv=False):
        """Returns (misfit, gradient[np + 2])."""
        pv = _host_vec(p, self.np)
        J = ctypes.c_double(0.0)
        g = np.zeros(self.np + 2)
        self.last_theta = None
        self._call(lib().rd_gradient(self.h, pv.ctypes.data, float(k_f), float(rho_f), ctypes.byref(J),
                                     g.ctypes.data), allow_noconv)
        self._remember(pv, k_f, rho_f)
        return J.value, g

    def rd_hessvec(self, p, k_f, rho_f, v, allow_noconv=False):
        pv = _host_vec(p, self.np)
        vv = _host_vec(v, self.np + 2)
        hv = np.zeros(self.np + 2)
        self.last_theta = None
        self._call(lib().rd_hessvec(self.h, pv.ctypes.data, float(k_f), float(rho_f), vv.ctypes.data,
                                    hv.ctypes.data), allow_noconv)
        self._remember(pv, k_f, rho_f)
        return hv

    def rd_apply_operator(self, k_f, u, out):
        (a, ka), (b, kb) = _ptr(u), _ptr(out)
        self._call(lib().rd_apply_operator(self.h, float(k_f), a, b))
        return out

    def rd_apply_precond(self, k_f, r, out):
        (a, ka), (b, kb) = _ptr(r), _ptr(out)
        self._call(lib().rd_apply_precond(self.h, float(k_f), a, b))
        return out

    def rd_active_tiles(self):
        """{"axis0": (active, all), "axis1": (...), "rows": (...)}: tiles of the
        operator passes where kappa1 is not identically zero."""
        c = (ctypes.c_longlong * 6)()
        self._call(lib().rd_active_tiles(self.h, c))
        return {"axis0": (c[0], c[1]), "axis1": (c[2], c[3]), "rows": (c[4], c[5])}

    def rd_last_pcg_iters(self):
        return lib().rd_last_pcg_iters(self.h)

    def rd_autotune(self, reps=3):
        """Tune tile shape and grid size per kernel class on this grid;
        returns {class: (blocks (0 = all resident), "pencil" | "tma")}."""
        n = 10
        caps = (ctypes.c_int * n)()
        pen = (ctypes.c_int * n)()
        self._call(lib().rd_autotune(self.h, int(reps), caps, pen, n))
        return {lib().rd_profile_class(i).decode(): (caps[i], "pencil" if pen[i] else "tma") for i in range(n)}

    def rd_last_graph_solves(self):
        return lib().rd_last_graph_solves(self.h)

    def rd_last_pcg_solves(self):
        return lib().rd_last_pcg_solves(self.h)

    def rd_last_error(self):
        return lib().rd_last_error(self.h).decode()


def rd_batch_gradient(ctxs, thetas, allow_noconv=False):
    """Gradients of several contexts in one graph launch.  thetas: list of
    (p, k_f, rho_f).  Returns (misfits, gradients)."""
    n = len(ctxs)
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in ctxs])
    ps = [_host_vec(t[0], c.np) for c, t in zip(ctxs, thetas)]
    gs = [np.zeros(c.np + 2) for c in ctxs]
    pp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in ps])
    gp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in gs])
    kf = (ctypes.c_double * n)(*[float(t[1]) for t in thetas])
    rf = (ctypes.c_double * n)(*[float(t[2]) for t in thetas])
    J = (ctypes.c_double * n)()
    status = lib().rd_batch_gradient(hs, n, pp, kf, rf, J, gp)
    if status != RD_OK and not (status == RD_ERR_NOCONV and allow_noconv):
        raise RDError(status, ctxs[0].rd_last_error())
    for c, t in zip(ctxs, thetas):
        c._remember(t[0], t[1], t[2])
    return list(J), gs


def context_for(prob, prec="fp64", **kw):
    """Context with tissue and basis set from a :class:`synth.Problem`."""
    ctx = Context(prob.n, prob.nt, len(prob.p), prec=prec, k_w=prob.k_w, rho_w=prob.rho_w, **kw)
    ctx.rd_set_tissue(prob.m_wm, prob.m_gm, prob.m_csf)
    ctx.rd_set_basis(prob.centers, prob.sigma)
    return ctx
