"""ctypes binding of the C ABI in include/ras.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libras.so``; this module
only converts torch tensors to device pointers and Python values to the ABI's
structs. It fails loudly if the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libras.so")

RAS_OK, RAS_GMRES_MAXIT, RAS_NEWTON_MAXIT, RAS_LINESEARCH_FAIL = 0, 1, 2, 3
RAS_EINVAL, RAS_ECUDA, RAS_ENOMEM, RAS_ENAN, RAS_EZEROPIVOT = -1, -2, -3, -4, -5
RAS_ENOROOT, RAS_ETIMEOUT = -6, -7

EXPORTED = ["ras_problem_create", "ras_problem_destroy", "residual_eval", "ras_stencil_matvec",
            "ras_setup", "ras_precond_destroy", "ras_factor", "ras_apply", "gmres_solve",
            "newton_step", "ras_status_string", "ras_last_error", "ras_kernel_launches",
            "ras_timing_enable", "ras_timing_read", "ras_apply_bytes", "ras_norm2_noalloc",
            "ras_stencil_transpose", "ras_adjoint_rhs", "ras_grad_logk", "ras_batch_create",
            "ras_batch_destroy", "ras_batch_gmres", "ras_batch_newton_step", "ras_set_apply_schedule",
            "ras_get_apply_schedule", "ras_set_apply_kernel", "ras_get_apply_kernel", "ras_gemm_f32",
            "ras_coarse_cr_schedule"]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double), ("gz", C.c_double),
                ("upwind", C.c_int), ("conservative", C.c_int)]


class Eos(C.Structure):
    _fields_ = [("Tc", C.c_double), ("pc", C.c_double), ("omega", C.c_double), ("Tb", C.c_double),
                ("omega_from_Tb", C.c_int), ("T", C.c_double), ("R", C.c_double),
                ("W", C.c_double), ("mu", C.c_double)]


class Rock(C.Structure):
    _fields_ = [("kx", C.c_void_p), ("ky", C.c_void_p), ("kz", C.c_void_p), ("phi", C.c_void_p),
                ("nconn", C.c_int), ("conn_cell", C.c_void_p), ("conn_p", C.c_void_p),
                ("conn_T", C.c_void_p), ("rate_Q", C.c_void_p)]


class Stencil(C.Structure):
    _fields_ = [("c", C.c_void_p * 7)]


class Opts(C.Structure):
    _fields_ = [("px", C.c_int), ("py", C.c_int), ("pz", C.c_int), ("overlap", C.c_int),
                ("ras_type", C.c_int), ("ilu_k", C.c_int), ("factor_prec", C.c_int),
                ("nlevels", C.c_int), ("coarsen", C.c_int * 3), ("interp_order", C.c_int),
                ("mlevel_type", C.c_int), ("coarse_prec", C.c_int), ("coarse_overlap", C.c_int),
                ("coarse_solver", C.c_int), ("coarse_rtol", C.c_double)]


class KrylovOpts(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("rtol", C.c_double),
                ("atol", C.c_double)]


class KrylovStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("r0", C.c_double),
                ("rfinal", C.c_double), ("history", C.POINTER(C.c_double)),
                ("history_cap", C.c_int), ("history_len", C.c_int)]


class NewtonOpts(C.Structure):
    _fields_ = [("maxit", C.c_int), ("rtol", C.c_double), ("atol", C.c_double),
                ("ls_alpha", C.c_double), ("ls_min_lambda", C.c_double), ("lin", KrylovOpts)]


class NewtonStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("lin_iters", C.c_int), ("residual_evals", C.c_int),
                ("f0", C.c_double), ("ffinal", C.c_double),
                ("fhistory", C.POINTER(C.c_double)), ("fhistory_cap", C.c_int),
                ("fhistory_len", C.c_int), ("lin_history", C.POINTER(C.c_int)),
                ("lin_history_cap", C.c_int), ("lambdas", C.POINTER(C.c_double))]


_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libras.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        sig = {
            "ras_problem_create": (i, [C.POINTER(Grid), C.POINTER(Eos), C.POINTER(Rock), vp, C.POINTER(vp)]),
            "ras_problem_destroy": (None, [vp]),
            "residual_eval": (i, [vp, vp, vp, vp, d, i, vp, C.POINTER(Stencil), C.POINTER(d), vp]),
            "ras_stencil_matvec": (i, [vp, C.POINTER(Stencil), vp, vp, vp]),
            "ras_setup": (i, [vp, C.POINTER(Opts), C.POINTER(vp)]),
            "ras_precond_destroy": (None, [vp]),
            "ras_factor": (i, [vp, C.POINTER(Stencil), vp]),
            "ras_apply": (i, [vp, vp, vp, vp]),
            "gmres_solve": (i, [vp, C.POINTER(Stencil), vp, vp, vp, C.POINTER(KrylovOpts),
                                C.POINTER(KrylovStats), vp]),
            "newton_step": (i, [vp, vp, vp, vp, vp, d, i, C.POINTER(NewtonOpts),
                                C.POINTER(NewtonStats), vp]),
            "ras_status_string": (C.c_char_p, [i]),
            "ras_last_error": (C.c_char_p, []),
            "ras_kernel_launches": (C.c_longlong, []),
            "ras_timing_enable": (i, [vp, i]),
            "ras_timing_read": (i, [vp, C.POINTER(d), C.POINTER(C.c_longlong), i]),
            "ras_apply_bytes": (d, [vp]),
            "ras_norm2_noalloc": (i, [vp, C.c_longlong, vp, vp]),
            "ras_stencil_transpose": (i, [vp, C.POINTER(Stencil), C.POINTER(Stencil), vp]),
            "ras_adjoint_rhs": (i, [vp, vp, vp, vp, d, vp, vp, d, vp, vp]),
            "ras_grad_logk": (i, [vp, vp, vp, vp, vp]),
            "ras_set_apply_schedule": (i, [vp, i, i]),
            "ras_get_apply_schedule": (i, [vp, C.POINTER(i), C.POINTER(i)]),
            "ras_set_apply_kernel": (i, [vp, i]),
            "ras_get_apply_kernel": (i, [vp, C.POINTER(i)]),
            "ras_gemm_f32": (i, [i, i, i, C.c_float, vp, i, vp, i, C.c_float, vp, i, vp]),
            "ras_coarse_cr_schedule": (i, [i, C.POINTER(i), i, C.POINTER(i), i, C.POINTER(i), C.POINTER(i),
                                           C.POINTER(i)]),
            "ras_batch_create": (i, [i, vp, vp, C.POINTER(vp)]),
            "ras_batch_destroy": (None, [vp]),
            "ras_batch_gmres": (i, [vp, vp, vp, vp, C.POINTER(KrylovOpts), vp, vp]),
            "ras_batch_newton_step": (i, [vp, vp, vp, vp, vp, i, C.POINTER(NewtonOpts), vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RasError(RuntimeError):
    def __init__(self, status, what):
        msg = lib().ras_status_string(status).decode()
        last = lib().ras_last_error().decode()
        super().__init__(f"{what}: status {status} ({msg}){' - ' + last if last else ''}")
        self.status = status


def check(status, what, ok=(RAS_OK,)):
    if status not in ok:
        raise RasError(status, what)
    return status


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def stencil_struct(J):
    """J: list of 7 device tensors (centre, -x, +x, -y, +y, -z, +z)."""
    st = Stencil()
    for s in range(7):
        st.c[s] = J[s].data_ptr()
    return st


def norm2_noalloc(x, out, stream=None):
    """||x||_2 into the one-element device tensor `out`; allocates nothing
    (partial sums in the library's static device array)."""
    check(lib().ras_norm2_noalloc(_ptr(x), x.numel(), _ptr(out), _stream(stream)),
          "ras_norm2_noalloc")


def gemm_f32(A, B, C, alpha=1.0, beta=0.0, stream=None):
    """C = alpha A B + beta C (FP32 row-major device tensors) on the tensor cores."""
    m, k = A.shape
    n = B.shape[1]
    check(lib().ras_gemm_f32(m, n, k, float(alpha), _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                             float(beta), _ptr(C), C.stride(0), _stream(stream)), "ras_gemm_f32")


def coarse_cr_schedule(nb):
    """(fac, sol, nslot): the cyclic-reduction schedules for nb coarse blocks (host only)."""
    fl, sl, ns = C.c_int(0), C.c_int(0), C.c_int(0)
    lib().ras_coarse_cr_schedule(nb, None, 0, None, 0, C.byref(fl), C.byref(sl), C.byref(ns))
    fac, sol = (C.c_int * max(fl.value, 1))(), (C.c_int * max(sl.value, 1))()
    check(lib().ras_coarse_cr_schedule(nb, fac, fl.value, sol, sl.value, C.byref(fl), C.byref(sl), C.byref(ns)),
          "ras_coarse_cr_schedule")
    return list(fac[:fl.value]), list(sol[:sl.value]), ns.value


def kernel_launches() -> int:
    return int(lib().ras_kernel_launches())


class Problem:
    """ras_problem handle built from a synthetic.Reservoir."""

    def __init__(self, res, device="cuda"):
        g = res.grid
        self.res = res
        self.N = g.n
        self.shape = (g.nx, g.ny, g.nz)
        dev = torch.device(device)
        f64 = dict(dtype=torch.float64, device=dev)
        self._kx = torch.as_tensor(res.kx, **f64).contiguous()
        self._ky = torch.as_tensor(res.ky, **f64).contiguous()
        self._kz = torch.as_tensor(res.kz, **f64).contiguous()
        self._phi = torch.as_tensor(res.phi, **f64).contiguous()
        self._cc = torch.as_tensor(res.conns.cell, dtype=torch.int32, device=dev).contiguous()
        self._cp = torch.as_tensor(res.conns.p, **f64).contiguous()
        self._cT = torch.as_tensor(res.conns.T, **f64).contiguous()
        rq = getattr(res, "rate_Q", None)
        self._rq = None if rq is None else torch.as_tensor(rq, **f64).contiguous()
        fl = res.fluid
        grid = Grid(g.nx, g.ny, g.nz, g.hx, g.hy, g.hz, float(getattr(res, "gravity", 0.0)),
                    1 if getattr(res, "upwind", False) else 0,
                    1 if getattr(res, "conservative", False) else 0)
        eos = Eos(fl.Tc, fl.pc, 0.0 if fl.omega_from_Tb else fl.omega, fl.Tb,
                  1 if fl.omega_from_Tb else 0, fl.T, fl.R, fl.W, fl.mu)
        rock = Rock(self._kx.data_ptr(), self._ky.data_ptr(), self._kz.data_ptr(),
                    self._phi.data_ptr(), len(res.conns), self._cc.data_ptr(),
                    self._cp.data_ptr(), self._cT.data_ptr(),
                    self._rq.data_ptr() if self._rq is not None else None)
        h = C.c_void_p()
        check(lib().ras_problem_create(C.byref(grid), C.byref(eos), C.byref(rock), _stream(),
                                       C.byref(h)), "ras_problem_create")
        self.h = h
        self.J = [torch.zeros(self.N, **f64) for _ in range(7)]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ras_problem_destroy(self.h)
            self.h = None

    def residual_eval(self, p, p_l, p_lm1, dt, order, F, J=None, want_norm=False):
        Js = stencil_struct(J) if J is not None else None
        nrm = C.c_double(0.0)
        check(lib().residual_eval(self.h, _ptr(p), _ptr(p_l), _ptr(p_lm1) if p_lm1 is not None else None,
                                  float(dt), int(order), _ptr(F),
                                  C.byref(Js) if Js is not None else None,
                                  C.byref(nrm) if want_norm else None, _stream()),
              "residual_eval")
        return nrm.value if want_norm else None

    def stencil_transpose(self, J, JT):
        Js, JTs = stencil_struct(J), stencil_struct(JT)
        check(lib().ras_stencil_transpose(self.h, C.byref(Js), C.byref(JTs), _stream()),
              "ras_stencil_transpose")

    def adjoint_rhs(self, dphi, p1, lam1, c1, p2, lam2, c2, rhs):
        opt = lambda t: _ptr(t) if t is not None else None
        check(lib().ras_adjoint_rhs(self.h, opt(dphi), opt(p1), opt(lam1), float(c1), opt(p2),
                                    opt(lam2), float(c2), _ptr(rhs), _stream()), "ras_adjoint_rhs")

    def grad_logk(self, p, lam, grad):
        check(lib().ras_grad_logk(self.h, _ptr(p), _ptr(lam), _ptr(grad), _stream()),
              "ras_grad_logk")

    def matvec(self, J, x, y):
        Js = stencil_struct(J)
        check(lib().ras_stencil_matvec(self.h, C.byref(Js), _ptr(x), _ptr(y), _stream()),
              "ras_stencil_matvec")

    def gmres_solve(self, J, pc, b, x, restart=30, maxit=1000, rtol=1e-6, atol=0.0,
                    history_cap=4096):
        Js = stencil_struct(J)
        ko = KrylovOpts(restart, maxit, rtol, atol)
        hist = (C.c_double * history_cap)()
        ks = KrylovStats(0, 0, 0.0, 0.0, hist, history_cap, 0)
        st = lib().gmres_solve(self.h, C.byref(Js), pc.h, _ptr(b), _ptr(x), C.byref(ko),
                               C.byref(ks), _stream())
        check(st, "gmres_solve", ok=(RAS_OK, RAS_GMRES_MAXIT))
        return {"status": st, "iters": ks.iters, "converged": bool(ks.converged), "r0": ks.r0,
                "rfinal": ks.rfinal, "history": list(hist[:ks.history_len])}

    def newton_step(self, pc, p, p_l, p_lm1, dt, order, rtol=1e-6, atol=1e-10, maxit=50,
                    lin_rtol=1e-6, lin_atol=1e-8, restart=30, lin_maxit=2000, alpha=1e-4,
                    lam_min=1e-8):
        no = NewtonOpts(maxit, rtol, atol, alpha, lam_min, KrylovOpts(restart, lin_maxit, lin_rtol, lin_atol))
        cap = 256
        fh = (C.c_double * cap)()
        lh = (C.c_int * cap)()
        lams = (C.c_double * cap)()
        ns = NewtonStats(0, 0, 0, 0.0, 0.0, fh, cap, 0, lh, cap, lams)
        st = lib().newton_step(self.h, pc.h, _ptr(p), _ptr(p_l),
                               _ptr(p_lm1) if p_lm1 is not None else None, float(dt), int(order),
                               C.byref(no), C.byref(ns), _stream())
        check(st, "newton_step", ok=(RAS_OK, RAS_NEWTON_MAXIT, RAS_LINESEARCH_FAIL))
        k = ns.iters
        return {"status": st, "newton_iters": k, "lin_iters": list(lh[:k]),
                "fnorm_history": list(fh[:ns.fhistory_len]), "lambdas": list(lams[:k]),
                "lin_total": ns.lin_iters, "residual_evals": ns.residual_evals,
                "f0": ns.f0, "ffinal": ns.ffinal}


class Precond:
    """ras_precond handle (left-RAS; two-level combinations; three-level V-cycle)."""

    def __init__(self, prob: Problem, parts, overlap, factor_prec=64, nlevels=1,
                 coarsen=(2, 2, 2), mlevel_type=0, coarse_prec=64, interp_order=2,
                 coarse_overlap=1, ras_type=1, ilu_k=0, coarse_solver=0, coarse_rtol=0.2):
        o = Opts(parts[0], parts[1], parts[2], overlap, ras_type, ilu_k, factor_prec, nlevels,
                 (C.c_int * 3)(*coarsen), interp_order, mlevel_type, coarse_prec,
                 coarse_overlap, coarse_solver, coarse_rtol)
        h = C.c_void_p()
        check(lib().ras_setup(prob.h, C.byref(o), C.byref(h)), "ras_setup")
        self.h = h
        self.prob = prob

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ras_precond_destroy(self.h)
            self.h = None

    def factor(self, J):
        Js = stencil_struct(J)
        check(lib().ras_factor(self.h, C.byref(Js), _stream()), "ras_factor")

    def apply(self, r, z):
        check(lib().ras_apply(self.h, _ptr(r), _ptr(z), _stream()), "ras_apply")

    def timing(self, enable=True):
        check(lib().ras_timing_enable(self.h, 1 if enable else 0), "ras_timing_enable")

    def timing_read(self, reset=True):
        ms = C.c_double(0.0)
        n = C.c_longlong(0)
        check(lib().ras_timing_read(self.h, C.byref(ms), C.byref(n), 1 if reset else 0),
              "ras_timing_read")
        return ms.value, n.value

    def apply_bytes(self) -> float:
        return float(lib().ras_apply_bytes(self.h))

    def set_schedule(self, chunk_cells=0, threads=0):
        """Level schedule of the subdomain solves (performance only; 0 = default)."""
        check(lib().ras_set_apply_schedule(self.h, int(chunk_cells), int(threads)), "ras_set_apply_schedule")

    def schedule(self):
        c, t = C.c_int(0), C.c_int(0)
        check(lib().ras_get_apply_schedule(self.h, C.byref(c), C.byref(t)), "ras_get_apply_schedule")
        return c.value, t.value

    def set_apply_kernel(self, kernel):
        """0: level-scheduled subdomain solves, 1: pencil-wavefront (same values from the same factors)."""
        check(lib().ras_set_apply_kernel(self.h, int(kernel)), "ras_set_apply_kernel")

    def apply_kernel(self):
        k = C.c_int(0)
        check(lib().ras_get_apply_kernel(self.h, C.byref(k)), "ras_get_apply_kernel")
        return k.value


class BatchSolver:
    """ras_batch handle: independent reservoirs whose FGMRES operations run in one
    launch each (one-level left-RAS preconditioners of one factor precision)."""

    def __init__(self, problems, preconds):
        n = len(problems)
        hp = (C.c_void_p * n)(*[q.h.value for q in problems])
        hc = (C.c_void_p * n)(*[q.h.value for q in preconds])
        h = C.c_void_p()
        check(lib().ras_batch_create(n, hp, hc, C.byref(h)), "ras_batch_create")
        self.h = h
        self.n = n
        self.problems, self.preconds = list(problems), list(preconds)   # must outlive the batch

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ras_batch_destroy(self.h)
            self.h = None

    @staticmethod
    def _ptrs(ts):
        return (C.c_void_p * len(ts))(*[_ptr(t) if t is not None else None for t in ts])

    def gmres(self, Js, bs, xs, restart=30, maxit=1000, rtol=1e-6, atol=0.0, history_cap=4096):
        n = self.n
        J = (Stencil * n)(*[stencil_struct(j) for j in Js])
        ko = KrylovOpts(restart, maxit, rtol, atol)
        hists = [(C.c_double * history_cap)() for _ in range(n)]
        ks = (KrylovStats * n)(*[KrylovStats(0, 0, 0.0, 0.0, h, history_cap, 0) for h in hists])
        st = lib().ras_batch_gmres(self.h, J, self._ptrs(bs), self._ptrs(xs), C.byref(ko), ks, _stream())
        check(st, "ras_batch_gmres", ok=(RAS_OK, RAS_GMRES_MAXIT))
        return [{"iters": k.iters, "converged": bool(k.converged), "r0": k.r0, "rfinal": k.rfinal,
                 "history": list(h[:k.history_len])} for k, h in zip(ks, hists)]

    def newton_step(self, ps, p_ls, p_lm1s, dts, order, rtol=1e-6, atol=1e-10, maxit=50,
                    lin_rtol=1e-6, lin_atol=1e-8, restart=30, lin_maxit=2000, alpha=1e-4,
                    lam_min=1e-8):
        n = self.n
        no = NewtonOpts(maxit, rtol, atol, alpha, lam_min, KrylovOpts(restart, lin_maxit, lin_rtol, lin_atol))
        cap = 256
        fh = [(C.c_double * cap)() for _ in range(n)]
        lh = [(C.c_int * cap)() for _ in range(n)]
        lams = [(C.c_double * cap)() for _ in range(n)]
        ns = (NewtonStats * n)(*[NewtonStats(0, 0, 0, 0.0, 0.0, fh[i], cap, 0, lh[i], cap, lams[i])
                                  for i in range(n)])
        dt = (C.c_double * n)(*[float(v) for v in dts])
        st = lib().ras_batch_newton_step(self.h, self._ptrs(ps), self._ptrs(p_ls),
                                         self._ptrs(p_lm1s) if p_lm1s is not None else None, dt,
                                         int(order), C.byref(no), ns, _stream())
        check(st, "ras_batch_newton_step", ok=(RAS_OK, RAS_NEWTON_MAXIT, RAS_LINESEARCH_FAIL))
        out = []
        for i in range(n):
            k = ns[i].iters
            out.append({"newton_iters": k, "lin_iters": list(lh[i][:k]),
                        "fnorm_history": list(fh[i][:ns[i].fhistory_len]), "lambdas": list(lams[i][:k]),
                        "lin_total": ns[i].lin_iters, "residual_evals": ns[i].residual_evals,
                        "f0": ns[i].f0, "ffinal": ns[i].ffinal})
        return st, out
