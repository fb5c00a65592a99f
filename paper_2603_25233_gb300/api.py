"""Python binding of the RTE library: the names of the C ABI (include/rte.h) over torch
device tensors and the caller's CUDA stream.  Argument marshalling only; every step of the
computation runs in the library's CUDA kernels.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_check(t, dtype, numel=None, name="tensor"):
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")


def default_opts(**kw):
    o = L.RteOpts()
    L.load().rte_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "mode":
            v = {"fr": L.RTE_MODE_FR, "lr": L.RTE_MODE_LR}.get(v, v)
        if k in ("sweep_precision", "dsa_precision", "basis_precision"):
            v = {"fp64": L.RTE_FP64, "fp32": L.RTE_FP32, "dw": L.RTE_DWF32}.get(v, v)
        if k == "mgs_test":
            v = {"first": 0, "max": 1}.get(v, v)
        if k == "sampling":
            v = {"residual": 0, "deim": 1}.get(v, v)
        if k == "basis_update":
            v = {"mgs2a": 0, "mgsqr": 1, "qr": 2}.get(v, v)
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class _DeviceView:
    """__cuda_array_interface__ view of library-owned float64 device memory."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}


class Handle:
    """One problem on the current CUDA device (rte_setup / rte_destroy)."""

    def __init__(self, spec, stream=None):
        self.lib = L.load()
        self.nx, self.ny = int(spec.nx), int(spec.ny)
        self._keep = []

        def dptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

        p = L.RteProblem()
        p.nx, p.ny = self.nx, self.ny
        p.x0, p.x1, p.y0, p.y1 = float(spec.x0), float(spec.x1), float(spec.y0), float(spec.y1)
        p.n_theta, p.n_omz = int(spec.n_theta), int(spec.n_omz)
        p.sig_t = dptr(spec.sig_t)
        p.sig_s = dptr(spec.sig_s)
        p.q_cell = dptr(spec.q_cell)
        rects = np.asarray(spec.q_rects, dtype=np.float64).reshape(-1, 5) if len(spec.q_rects) else None
        p.n_rect = 0 if rects is None else rects.shape[0]
        p.q_rects = dptr(rects)
        for k in range(4):
            p.inflow[k] = float(spec.inflow[k])
        gauss = getattr(spec, "q_gauss", None)
        gauss = np.asarray(gauss, dtype=np.float64).reshape(-1, 4) if gauss is not None and len(gauss) else None
        p.n_gauss = 0 if gauss is None else gauss.shape[0]
        p.q_gauss = dptr(gauss)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        L.check(self.lib.rte_setup(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        nd, nc, na = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(self.lib.rte_get_sizes(h, ctypes.byref(nd), ctypes.byref(nc), ctypes.byref(na)))
        self.n_dof, self.n_cells, self.n_angles = nd.value, nc.value, na.value
        self._keep = []

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.rte_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- data ----------------------------------------------------------------
    def set_materials(self, sig_t, sig_s, q_cell=None):
        st = np.ascontiguousarray(sig_t, dtype=np.float64)
        ss = np.ascontiguousarray(sig_s, dtype=np.float64)
        qc = None if q_cell is None else np.ascontiguousarray(q_cell, dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        L.check(self.lib.rte_set_materials(self.h, st.ctypes.data_as(dp), ss.ctypes.data_as(dp),
                                           None if qc is None else qc.ctypes.data_as(dp)))

    def set_wait_limit(self, spins):
        """rte_set_wait_limit: polls of a sweep hand-off wait before it gives up (0 = default)."""
        L.check(self.lib.rte_set_wait_limit(self.h, int(spins)))

    @staticmethod
    def _sprec(precision):
        return {"fp64": L.RTE_FP64, "fp32": L.RTE_FP32}.get(precision, precision)

    def sweep_tune(self, precision, n, with_psi=True):
        """rte_sweep_tune: time every valid sweep configuration for n-ordinate launches now and
        keep the fastest; returns it as a dict (kernel, warps, depth, staged, angles_per_block, ms)."""
        c = L.RteSweepConfig()
        L.check(self.lib.rte_sweep_tune(self.h, self._sprec(precision), int(n), int(bool(with_psi)), ctypes.byref(c)))
        return c.as_dict()

    def sweep_set_config(self, precision, n, with_psi=True, config=None):
        """rte_sweep_set_config: force a configuration (dict as returned by sweep_tune), or forget
        it (config=None)."""
        ptr = None
        if config is not None:
            kind = {"band": L.RTE_SWEEP_BAND, "warp": L.RTE_SWEEP_WARP}.get(config["kernel"], config["kernel"])
            c = L.RteSweepConfig(kind, int(config.get("warps", 0)), int(config.get("depth", 0)),
                                 int(config.get("staged", 0)), int(config.get("angles_per_block", 1)), 0.0)
            ptr = ctypes.byref(c)
        L.check(self.lib.rte_sweep_set_config(self.h, self._sprec(precision), int(n), int(bool(with_psi)), ptr))

    def sweep_get_config(self, precision, n, with_psi=True):
        """rte_sweep_get_config: the configuration n-ordinate launches use now."""
        c = L.RteSweepConfig()
        L.check(self.lib.rte_sweep_get_config(self.h, self._sprec(precision), int(n), int(bool(with_psi)),
                                              ctypes.byref(c)))
        return c.as_dict()

    def inject_failure(self, code):
        """rte_inject_failure (tests): the next low-rank solve reports `code` (RTE_ERR_SINGULAR)."""
        L.check(self.lib.rte_inject_failure(self.h, int(code)))

    def quadrature(self):
        out = [np.zeros(self.n_angles) for _ in range(4)]
        dp = ctypes.POINTER(ctypes.c_double)
        L.check(self.lib.rte_get_quadrature(self.h, *[a.ctypes.data_as(dp) for a in out]))
        return tuple(out)

    def source(self):
        G = torch.empty(self.n_dof, dtype=torch.float64, device="cuda")
        L.check(self.lib.rte_get_source(self.h, _ptr(G)))
        return G

    # -- compute -------------------------------------------------------------
    def _sweep(self, fn, angles, src, precision, src_per_angle, extra, psi_out, phi_out):
        ang = np.ascontiguousarray(angles, dtype=np.int32)
        dt = torch.float32 if precision == L.RTE_FP32 else torch.float64
        n = len(ang)
        _dev_check(src, dt, (n if src_per_angle else 1) * self.n_dof, "src")
        _dev_check(psi_out, dt, n * self.n_dof, "psi_out")
        _dev_check(phi_out, torch.float64, self.n_dof, "phi_out")
        ip = ang.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        L.check(fn(self.h, ip, n, precision, _ptr(src), int(src_per_angle), *extra, _ptr(psi_out), _ptr(phi_out)))

    def sweep(self, angles, src, precision=L.RTE_FP64, src_per_angle=False, add_inflow=True,
              psi_out=None, phi_out=None):
        """rte_sweep: psi_j = (D_j + Sigma_t)^{-1}(src + g_j^bc) for the listed angles."""
        self._sweep(self.lib.rte_sweep, angles, src, precision, src_per_angle, (int(add_inflow),), psi_out, phi_out)

    def sweep_adjoint(self, angles, src, precision=L.RTE_FP64, src_per_angle=False, mu_out=None, chi_out=None):
        """rte_sweep_adjoint: (D_j + Sigma_t)^T mu_j = src for the listed angles."""
        self._sweep(self.lib.rte_sweep_adjoint, angles, src, precision, src_per_angle, (), mu_out, chi_out)

    def si_dsa_solve(self, opts=None, phi=None, **kw):
        """rte_si_dsa_solve; returns (phi, stats dict).  Raises on any status but
        RTE_ERR_NOT_CONVERGED (reported in the stats)."""
        o = opts if isinstance(opts, L.RteOpts) else default_opts(**(opts or {}), **kw)
        if phi is None:
            phi = torch.zeros(self.n_dof, dtype=torch.float64, device="cuda")
        _dev_check(phi, torch.float64, self.n_dof, "phi")
        s = L.RteStats()
        rc = self.lib.rte_si_dsa_solve(self.h, ctypes.byref(o), _ptr(phi), ctypes.byref(s))
        if rc not in (L.RTE_OK, L.RTE_ERR_NOT_CONVERGED):
            L.check(rc)
        return phi, s.as_dict()

    def be_step(self, dt, psi_prev, phi=None, psi_next=None, opts=None, **kw):
        """rte_be_step: one backward-Euler step of length dt from psi_prev (float64 CUDA tensor
        [N_Omega * N_x], ordinate-major); returns (phi^{n+1}, psi^{n+1}, stats dict).  phi, when
        given, is the initial guess and receives the result."""
        o = opts if isinstance(opts, L.RteOpts) else default_opts(**(opts or {}), **kw)
        n = self.n_angles * self.n_dof
        _dev_check(psi_prev, torch.float64, n, "psi_prev")
        if phi is None:
            phi = torch.zeros(self.n_dof, dtype=torch.float64, device="cuda")
        _dev_check(phi, torch.float64, self.n_dof, "phi")
        if psi_next is None:
            psi_next = torch.empty(n, dtype=torch.float64, device="cuda")
        _dev_check(psi_next, torch.float64, n, "psi_next")
        s = L.RteStats()
        rc = self.lib.rte_be_step(self.h, ctypes.byref(o), float(dt), _ptr(psi_prev), _ptr(psi_next), _ptr(phi),
                                  ctypes.byref(s))
        if rc not in (L.RTE_OK, L.RTE_ERR_NOT_CONVERGED):
            L.check(rc)
        return phi, psi_next, s.as_dict()

    def lowrank_state(self):
        """rte_get_lowrank_state: copies of the last low-rank solve's basis X [N_x, r] and its
        projected operators X^T D_x^- X, X^T D_y^- X, X^T Sigma_t X [r, r] as torch tensors."""
        r, ld = ctypes.c_int(), ctypes.c_int()
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        L.check(self.lib.rte_get_lowrank_state(self.h, ctypes.byref(r), ctypes.byref(ld),
                                               *[ctypes.byref(p) for p in ptrs]))
        rk, n = r.value, ld.value

        def view(ptr, shape):
            return torch.as_tensor(_DeviceView(ptr, shape), device="cuda").clone()

        X = view(ptrs[0].value, (rk, self.n_dof)).T.contiguous()
        ops = [view(p.value, (n, n))[:rk, :rk].T.contiguous() for p in ptrs[1:]]   # (i, k) at [k * ld + i]
        return {"X": X, "Pxm": ops[0], "Pym": ops[1], "T": ops[2]}

    def factors(self):
        """rte_get_factors: copies of X [N_x, r'], S [r'], V [N_Omega, r'] as torch tensors."""
        X, S, V, r = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int()
        L.check(self.lib.rte_get_factors(self.h, ctypes.byref(X), ctypes.byref(S), ctypes.byref(V), ctypes.byref(r)))
        rk = r.value

        def view(ptr, shape):
            return torch.as_tensor(_DeviceView(ptr, shape), device="cuda").clone()

        Xt = view(X.value, (rk, self.n_dof)).T.contiguous()
        Vt = view(V.value, (rk, self.n_angles)).T.contiguous()
        return Xt, view(S.value, (rk,)), Vt

    def adjoint_grad(self, phi, det, opts=None, **kw):
        o = opts if isinstance(opts, L.RteOpts) else default_opts(**(opts or {}), **kw)
        _dev_check(phi, torch.float64, self.n_dof, "phi")
        _dev_check(det, torch.float64, self.n_dof, "det")
        gt = torch.empty(self.n_cells, dtype=torch.float64, device="cuda")
        gs = torch.empty_like(gt)
        gq = torch.empty_like(gt)
        s = L.RteStats()
        L.check(self.lib.rte_adjoint_grad(self.h, ctypes.byref(o), _ptr(phi), _ptr(det), _ptr(gt), _ptr(gs),
                                          _ptr(gq), ctypes.byref(s)))
        return dict(sig_t=gt, sig_s=gs, q=gq, stats=s.as_dict())

    def basis_project(self, X, Psi):
        """rte_basis_project: X^T Psi on the tensor cores (split TF32) for float32 CUDA tensors X
        [r, N_x] (basis columns as rows) and Psi [nv, N_x]; returns float64 [nv, r]."""
        _dev_check(X, torch.float32, None, "X")
        _dev_check(Psi, torch.float32, None, "Psi")
        r, nv = X.shape[0], Psi.shape[0]
        if X.shape[1] != self.n_dof or Psi.shape[1] != self.n_dof:
            raise ValueError("X and Psi rows must have the handle's DOF length")
        out = torch.empty(nv * r, dtype=torch.float64, device="cuda")
        L.check(self.lib.rte_basis_project(self.h, _ptr(X), r, _ptr(Psi), nv, _ptr(out)))
        return out.reshape(nv, r)

    def dsa_apply(self, x, y=None):
        _dev_check(x, torch.float64, self.n_dof, "x")
        y = torch.empty_like(x) if y is None else y
        L.check(self.lib.rte_dsa_apply(self.h, _ptr(x), _ptr(y)))
        return y

    def dsa_solve(self, rhs, tol=1e-12, max_iter=20000, x=None):
        _dev_check(rhs, torch.float64, self.n_dof, "rhs")
        x = torch.empty_like(rhs) if x is None else x
        it = ctypes.c_int()
        L.check(self.lib.rte_dsa_solve(self.h, _ptr(rhs), _ptr(x), float(tol), int(max_iter), ctypes.byref(it)))
        return x, it.value

    # -- instrumentation ------------------------------------------------------
    def profile_enable(self, on=True):
        """rte_profile_enable: start (and zero) or stop per-kernel-class CUDA-event timing."""
        L.check(self.lib.rte_profile_enable(self.h, int(bool(on))))

    def profile_read(self):
        """rte_profile_read for every class: {name: dict(ms, launches, bytes, flops)}."""
        out = {}
        for name, cls in L.PROF_CLASSES.items():
            ms, n, by, fl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
            L.check(self.lib.rte_profile_read(self.h, cls, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by),
                                              ctypes.byref(fl)))
            out[name] = dict(ms=ms.value, launches=n.value, bytes=by.value, flops=fl.value)
        return out


def sweep_batch(handles, angles, srcs, precision=L.RTE_FP64, add_inflow=True, psi_outs=None):
    """rte_sweep_batch: the sweeps of several problems (handles[i], angles[i], srcs[i]) in one
    launch; returns the list of psi tensors [len(angles[i]) * N_x_i]."""
    lib = L.load()
    n = len(handles)
    if not (len(angles) == len(srcs) == n) or n == 0:
        raise ValueError("handles, angles and srcs must be non-empty lists of equal length")
    dt = torch.float32 if precision == L.RTE_FP32 else torch.float64
    angs = [np.ascontiguousarray(a, dtype=np.int32) for a in angles]
    if psi_outs is None:
        psi_outs = [torch.empty(len(a) * h.n_dof, dtype=dt, device="cuda") for h, a in zip(handles, angs)]
    for h, a, s, o in zip(handles, angs, srcs, psi_outs):
        _dev_check(s, dt, h.n_dof, "src")
        _dev_check(o, dt, len(a) * h.n_dof, "psi_out")
    ip = ctypes.POINTER(ctypes.c_int)
    hs = (ctypes.c_void_p * n)(*[h.h.value for h in handles])
    al = (ip * n)(*[a.ctypes.data_as(ip) for a in angs])
    na = (ctypes.c_int * n)(*[len(a) for a in angs])
    sp = (ctypes.c_void_p * n)(*[s.data_ptr() for s in srcs])
    op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in psi_outs])
    L.check(lib.rte_sweep_batch(hs, n, al, na, precision, sp, int(add_inflow), op))
    return psi_outs


def si_dsa_solve_batch(handles, opts=None, phis=None, **kw):
    """rte_si_dsa_solve_batch (full rank in lock step, or low rank with the problems' solves
    running concurrently): returns (list of phi, list of stats dicts).  Raises on any status but
    RTE_ERR_NOT_CONVERGED (reported per problem in the stats)."""
    lib = L.load()
    o = opts if isinstance(opts, L.RteOpts) else default_opts(**(opts or {}), **kw)
    n = len(handles)
    if phis is None:
        phis = [torch.zeros(h.n_dof, dtype=torch.float64, device="cuda") for h in handles]
    for h, p in zip(handles, phis):
        _dev_check(p, torch.float64, h.n_dof, "phi")
    hs = (ctypes.c_void_p * n)(*[h.h.value for h in handles])
    pp = (ctypes.c_void_p * n)(*[p.data_ptr() for p in phis])
    st = (L.RteStats * n)()
    rc = lib.rte_si_dsa_solve_batch(hs, n, ctypes.byref(o), pp, st)
    if rc not in (L.RTE_OK, L.RTE_ERR_NOT_CONVERGED):
        L.check(rc)
    return phis, [s.as_dict() for s in st]


class RTEResponse(torch.autograd.Function):
    """Detector response R = d . phi(sigma_t, sigma_s, q) of the converged SI-DSA solution, with
    gradients from the library's discrete adjoint (rte_adjoint_grad).

    forward(sig_t, sig_s, q, handle, det, opts): sig_t, sig_s, q are float64 tensors [n_cells]
    (per-cell total and scattering cross sections and a per-cell constant source added to the
    handle's rectangles); det is a float64 CUDA tensor [N_x] (e.g. exact overlap integrals of
    a detector rectangle).  Nothing of the angular flux is stored between forward and backward:
    the backward pass regenerates psi_j by one sweep from the converged phi and contracts it with
    the adjoint sweeps on the fly.
    """

    @staticmethod
    def forward(ctx, sig_t, sig_s, q, handle, det, opts):
        to_np = lambda t: t.detach().double().cpu().numpy()
        handle.set_materials(to_np(sig_t), to_np(sig_s), to_np(q))
        phi, st = handle.si_dsa_solve(dict(opts))
        if not st["converged"]:
            raise L.RteError(L.RTE_ERR_NOT_CONVERGED, "forward SI-DSA did not converge")
        ctx.save_for_backward(phi, det)
        ctx.handle = handle
        ctx.opts = dict(opts)
        ctx.devs = (sig_t.device, sig_s.device, q.device)
        return torch.dot(det, phi).reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        phi, det = ctx.saved_tensors
        opts = {k: v for k, v in ctx.opts.items() if k not in ("mode", "want_factors")}
        g = ctx.handle.adjoint_grad(phi, det, **opts)
        go = grad_out.to(phi.device)
        return (
            (go * g["sig_t"]).to(ctx.devs[0]),
            (go * g["sig_s"]).to(ctx.devs[1]),
            (go * g["q"]).to(ctx.devs[2]),
            None, None, None,
        )


def detector_response(handle, sig_t, sig_s, q, det, **opts):
    """Differentiable R = d . phi (see RTEResponse)."""
    return RTEResponse.apply(sig_t, sig_s, q, handle, det, opts)
