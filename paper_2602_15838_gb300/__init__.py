"""Python binding of libtadmm (GB300 batched ADMM for multi-agent trajectory QPs).

Argument marshalling only: every step of the solver runs in the CUDA kernels of
libtadmm.so, reached through its C ABI (include/tadmm.h).  PyTorch supplies the
current CUDA stream and device tensors for results.  There is no CPU fallback:
if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtadmm.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE = 0, -1, -2, -3, -4
CONVERGED, NOT_CONVERGED, QP_FAIL, NUMERIC = 0, 1, 2, 3
START = {"cold": 0, "hot": 1, "turbo": 2, "homotopy": 3}
FLAG_NO_FUSED_PAIR_GATHER, FLAG_NO_STRUCTURE, FLAG_NO_GROUPING, FLAG_DOUBLE_FLOAT = 1, 2, 4, 8
FLAG_NO_LANE_GROUPS = FLAG_NO_COOP_REFACTOR = 16
MODE = {"batched": 0, "plain": 1, "graph": 2}

_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


class TadmmBatch(C.Structure):
    _fields_ = [("n_scen", C.c_int32), ("nx", C.c_int32), ("nu", C.c_int32), ("dp", C.c_int32),
                ("N", _i32p), ("T", _i32p), ("A", _dp), ("B", _dp), ("umin", _dp), ("umax", _dp),
                ("Qd", _dp), ("Rd", _dp), ("Qfd", _dp), ("x_init", _dp), ("x_ref", _dp), ("a", _dp),
                ("w0", _dp), ("d_min", _dp), ("rho", _dp), ("pair_count", _i32p), ("pair_ij", _i32p),
                ("A_agent", _dp), ("B_agent", _dp)]


class TadmmOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("start_mode", C.c_int32), ("as_max", C.c_int32),
                ("eps_rel", C.c_double), ("mode", C.c_int32), ("threads_per_cta", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("kernel_variant", C.c_int32), ("flags", C.c_int32),
                ("adapt_every", C.c_int32), ("adapt_mu", C.c_double), ("adapt_tau", C.c_double),
                ("relax_alpha", C.c_double)]


class TadmmError(RuntimeError):
    pass


_LIB = None


def lib():
    """Loads libtadmm.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise TadmmError(f"{LIB_PATH} is missing: build it with paper_2602_15838_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        L.tadmm_create.argtypes = [C.POINTER(TadmmBatch), C.POINTER(TadmmOptions), C.POINTER(C.c_void_p)]
        L.tadmm_update.argtypes = [C.c_void_p, C.POINTER(TadmmBatch), C.c_void_p]
        L.tadmm_solve.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.c_void_p]
        L.tadmm_update_costs.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.tadmm_get_solution.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
        L.tadmm_get_counters.argtypes = [C.c_void_p, _i64p, _i64p, _i64p]
        L.tadmm_get_penalty.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
        L.tadmm_relinearize.argtypes = [C.c_void_p, C.c_void_p]
        L.tadmm_sqp.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_double, _i32p, _i32p,
                                C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]
        L.tadmm_autotune.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, _i32p, _i32p, _i32p]
        L.tadmm_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.tadmm_polish.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.c_double, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]
        L.tadmm_destroy.argtypes = [C.c_void_p]
        L.tadmm_destroy.restype = None
        L.tadmm_last_error.restype = C.c_char_p
        L.tadmm_version.restype = C.c_char_p
        _LIB = L
    return _LIB


def _check(rc: int, what: str):
    if rc != OK:
        msg = lib().tadmm_last_error().decode()
        raise TadmmError(f"{what} failed ({rc}): {msg}")


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _HostBatch:
    """Keeps the packed float64 arrays of an instance batch alive for a C call."""

    def __init__(self, batch, pinned: bool = False):
        fields = dict(A=batch.A, B=batch.B, umin=batch.umin, umax=batch.umax, Qd=batch.Qd, Rd=batch.Rd,
                      Qfd=batch.Qfd, x_init=batch.x_init, x_ref=batch.x_ref,
                      a=batch.a if batch.a.size else np.zeros((1, batch.dp)), w0=batch.w0,
                      d_min=batch.d_min, rho=batch.rho)
        hetero = getattr(batch, "A_agent", None) is not None
        if hetero:
            fields.update(A_agent=batch.A_agent, B_agent=batch.B_agent)
        self.keep = {k: _f64(v) for k, v in fields.items()}
        if pinned:
            import torch
            self.pinned = {k: torch.from_numpy(v).pin_memory() for k, v in self.keep.items()}
            ptr = {k: C.cast(C.c_void_p(t.data_ptr()), _dp) for k, t in self.pinned.items()}
        else:
            ptr = {k: v.ctypes.data_as(_dp) for k, v in self.keep.items()}
        self.N = np.ascontiguousarray(batch.N, dtype=np.int32)
        self.T = np.ascontiguousarray(batch.T, dtype=np.int32)
        listed = getattr(batch, "pair_ij", None) is not None
        self.pc = np.ascontiguousarray(batch.pair_count, dtype=np.int32) if listed else None
        self.pij = (np.ascontiguousarray(batch.pair_ij, dtype=np.int32).reshape(-1) if listed else None)
        if listed and self.pij.size == 0:
            self.pij = np.zeros(2, dtype=np.int32)
        self.s = TadmmBatch(int(batch.n_scen), batch.nx, batch.nu, batch.dp, self.N.ctypes.data_as(_i32p),
                            self.T.ctypes.data_as(_i32p), ptr["A"], ptr["B"], ptr["umin"], ptr["umax"],
                            ptr["Qd"], ptr["Rd"], ptr["Qfd"], ptr["x_init"], ptr["x_ref"],
                            None if not batch.a.size else ptr["a"], ptr["w0"], ptr["d_min"], ptr["rho"],
                            self.pc.ctypes.data_as(_i32p) if listed else None,
                            self.pij.ctypes.data_as(_i32p) if listed else None,
                            ptr["A_agent"] if hetero else None, ptr["B_agent"] if hetero else None)


class Solver:
    """A batch of scenarios resident on the current GPU (tadmm_create).

    precision: 64 or 32; start: 'turbo' | 'hot' | 'cold' | 'homotopy' (plain and
    graph modes); mode: 'batched' | 'plain' | 'graph'.  Results are float64 regardless of the arithmetic precision.
    """

    def __init__(self, batch, precision: int = 64, start: str = "turbo", mode: str = "batched",
                 as_max: int = 0, eps_rel: float = 0.0, threads_per_cta: int = 0, ctas_per_sm: int = 0,
                 kernel_variant: int = 0, flags: int = 0, adapt=None, relax: float = 1.0):
        """adapt = (every, mu, tau) turns on residual balancing of rho (batched mode);
        relax = alpha in (0, 2) over-relaxes the consensus and dual update (batched mode)."""
        import torch
        if not torch.cuda.is_available():
            raise TadmmError("no CUDA device: the solver has no CPU path")
        self.batch = batch
        self.precision = precision
        self._hb = _HostBatch(batch)
        ae, am, at = (0, 10.0, 2.0) if adapt is None else adapt
        opt = TadmmOptions(precision, START[start], as_max, eps_rel, MODE[mode], threads_per_cta, ctas_per_sm,
                           kernel_variant, flags, int(ae), float(am), float(at), float(relax))
        h = C.c_void_p()
        _check(lib().tadmm_create(C.byref(self._hb.s), C.byref(opt), C.byref(h)), "tadmm_create")
        self.h = h
        self.n_scen = int(batch.n_scen)
        self.sizes = dict(X=int((batch.N * (batch.T + 1)).sum()) * batch.nx,
                          U=int((batch.N * batch.T).sum()) * batch.nu,
                          theta=int((batch.P * batch.T).sum()))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                lib().tadmm_destroy(h)
            except Exception:
                pass
            self.h = None

    def close(self):
        self.__del__()

    def update(self, batch, stream=None, pinned_batch: Optional[_HostBatch] = None):
        hb = pinned_batch if pinned_batch is not None else _HostBatch(batch)
        self._upd = hb
        _check(lib().tadmm_update(self.h, C.byref(hb.s), C.c_void_p(_stream_ptr(stream))), "tadmm_update")

    def update_costs(self, Qd=None, Rd=None, Qfd=None, x_ref=None, stream=None):
        """Replaces diag Q, diag R, diag Qf and the goal states (tadmm_update_costs)
        from numpy arrays or float64 torch tensors (host or CUDA); None keeps an
        array.  The values are checked on the device."""
        keep = []

        def ptr(v, shape):
            if v is None:
                return None
            if hasattr(v, "data_ptr"):
                t = v.detach().to(dtype=__import__("torch").float64).contiguous()
                assert tuple(t.shape) == shape, (tuple(t.shape), shape)
                keep.append(t)
                return C.c_void_p(t.data_ptr())
            a = np.ascontiguousarray(v, dtype=np.float64).reshape(shape)
            keep.append(a)
            return C.c_void_p(a.ctypes.data)
        na, b = int(self.batch.N.sum()), self.batch
        _check(lib().tadmm_update_costs(self.h, ptr(Qd, (na, b.nx)), ptr(Rd, (na, b.nu)), ptr(Qfd, (na, b.nx)),
                                        ptr(x_ref, (na, b.nx)), C.c_void_p(_stream_ptr(stream))),
               "tadmm_update_costs")

    def polished_states(self, theta_eps: float = 1e-9, stream=None):
        """Polished states at the final (or polished) active set as a float64
        CUDA tensor in the packed layout of X (tadmm_backward without a loss
        gradient, writing straight to device memory)."""
        import torch
        X = torch.empty(self.sizes["X"], dtype=torch.float64, device="cuda")
        st = np.zeros(self.n_scen, dtype=np.int32)
        _check(lib().tadmm_backward(self.h, None, float(theta_eps), None, None, None, None, C.c_void_p(X.data_ptr()),
                                    C.c_void_p(st.ctypes.data), None, C.c_void_p(_stream_ptr(stream))),
               "tadmm_backward")
        return X, st

    def solve(self, tol: float = 1e-4, max_iter: int = 500, stream=None):
        _check(lib().tadmm_solve(self.h, float(tol), int(max_iter), C.c_void_p(_stream_ptr(stream))), "tadmm_solve")

    def autotune(self, probe_iter: int = 20, stream=None):
        """Returns the chosen (threads_per_cta, ctas_per_sm, kernel_variant)."""
        t = C.c_int32(0); c = C.c_int32(0); v = C.c_int32(0)
        _check(lib().tadmm_autotune(self.h, int(probe_iter), C.c_void_p(_stream_ptr(stream)), C.byref(t),
                                    C.byref(c), C.byref(v)), "tadmm_autotune")
        return t.value, c.value, v.value

    def solution(self, device: bool = False, stream=None):
        """Results as numpy arrays (host) or float64 torch tensors on the GPU."""
        import torch
        b = self.batch
        if device:
            X = torch.empty(self.sizes["X"], dtype=torch.float64, device="cuda")
            U = torch.empty(self.sizes["U"], dtype=torch.float64, device="cuda")
            th = torch.empty(max(self.sizes["theta"], 1), dtype=torch.float64, device="cuda")
            W = torch.empty(self.sizes["U"], dtype=torch.int8, device="cuda")
            ptr = lambda t: C.c_void_p(t.data_ptr())
        else:
            X = np.zeros(self.sizes["X"]); U = np.zeros(self.sizes["U"])
            th = np.zeros(max(self.sizes["theta"], 1)); W = np.zeros(self.sizes["U"], dtype=np.int8)
            ptr = lambda a: C.c_void_p(a.ctypes.data)
        st = np.zeros(self.n_scen, dtype=np.int32)
        it = np.zeros(self.n_scen, dtype=np.int32)
        res = np.zeros((self.n_scen, 2))
        _check(lib().tadmm_get_solution(self.h, ptr(X), ptr(U), ptr(th) if self.sizes["theta"] else None, ptr(W),
                                        C.c_void_p(st.ctypes.data), C.c_void_p(it.ctypes.data),
                                        C.c_void_p(res.ctypes.data), C.c_void_p(_stream_ptr(stream))),
               "tadmm_get_solution")
        return dict(X=X, U=U, theta=th[:self.sizes["theta"]], W=W, status=st, iters=it, res=res)

    def backward(self, grad_X, theta_eps: float = 1e-9, polished: bool = True, stream=None):
        """Implicit-KKT gradients of a loss at the final active set of the last solve
        (or the set refined by polish()).

        grad_X: dl/dX in the packed layout of X (numpy array or CUDA tensor), or
        None for the polished states alone.  Returns numpy arrays gQ, gQf, gR,
        gGoal (per agent), the polished states X_polished, the per-scenario
        status and the number of active halfspace rows found linearly dependent
        (n_dependent)."""
        b = self.batch
        na = int(b.N.sum())
        if grad_X is None:
            keep = None
            gptr = None
        elif hasattr(grad_X, "data_ptr"):
            g = grad_X.detach().to(dtype=__import__("torch").float64).contiguous()
            gptr = C.c_void_p(g.data_ptr())
            keep = g
        else:
            keep = np.ascontiguousarray(grad_X, dtype=np.float64).reshape(-1)
            assert keep.size == self.sizes["X"]
            gptr = C.c_void_p(keep.ctypes.data)
        gQ = np.zeros((na, b.nx)); gQf = np.zeros((na, b.nx)); gR = np.zeros((na, b.nu)); gG = np.zeros((na, b.nx))
        Xp = np.zeros(self.sizes["X"]) if polished else None
        st = np.zeros(self.n_scen, dtype=np.int32)
        nd = np.zeros(self.n_scen, dtype=np.int32)
        p = lambda a: C.c_void_p(a.ctypes.data) if a is not None else None
        _check(lib().tadmm_backward(self.h, gptr, float(theta_eps), p(gQ), p(gQf), p(gR), p(gG), p(Xp),
                                    p(st), p(nd), C.c_void_p(_stream_ptr(stream))), "tadmm_backward")
        del keep
        return dict(gQ=gQ, gQf=gQf, gR=gR, gGoal=gG, X_polished=Xp, status=st, n_dependent=nd)

    def polish(self, theta_eps: float = 1e-9, max_rounds: int = 20, kkt_tol: float = 0.0, stream=None):
        """Refines the active set of the last solve on the centralized QP until
        the KKT conditions hold (tadmm_polish); backward() then uses it.
        Returns the halfspace flags act [sum P T] (pair-step order of `a`), the
        held inputs W [sum N T nu], the per-scenario status and the rounds."""
        act = np.zeros(max(self.sizes["theta"], 1), dtype=np.uint8)
        W = np.zeros(self.sizes["U"], dtype=np.int8)
        st = np.zeros(self.n_scen, dtype=np.int32)
        nr = C.c_int32(0)
        _check(lib().tadmm_polish(self.h, float(theta_eps), int(max_rounds), float(kkt_tol),
                                  C.c_void_p(act.ctypes.data), C.c_void_p(W.ctypes.data),
                                  C.c_void_p(st.ctypes.data), C.byref(nr), C.c_void_p(_stream_ptr(stream))),
               "tadmm_polish")
        return dict(act=act[:self.sizes["theta"]], W=W, status=st, rounds=nr.value)

    def counters(self):
        eqp = np.zeros(self.n_scen, dtype=np.int64)
        fact = np.zeros(self.n_scen, dtype=np.int64)
        ps = np.zeros(self.n_scen, dtype=np.int64)
        _check(lib().tadmm_get_counters(self.h, eqp.ctypes.data_as(_i64p), fact.ctypes.data_as(_i64p),
                                        ps.ctypes.data_as(_i64p)), "tadmm_get_counters")
        return dict(eqp=eqp, fact=fact, pairsteps=ps)

    def relinearize(self, stream=None):
        """Re-linearizes every scenario's collision halfspaces (and the initial
        consensus positions) at the last solution; the next solve() solves the
        new QP (one outer step of a linearize-and-solve loop)."""
        _check(lib().tadmm_relinearize(self.h, C.c_void_p(_stream_ptr(stream))), "tadmm_relinearize")

    def sqp(self, tol=1e-4, max_iter=500, max_outer=10, obj_rtol=1e-4, dist_tol=-1.0, stream=None):
        """Sequential linearize-and-solve loop with the termination rule of
        Sec. V.A (relative objective change <= obj_rtol between outer steps and
        every pair at least d_min - dist_tol apart; dist_tol < 0: 2 sqrt(dp) tol),
        at most max_outer steps.  Returns per-scenario numpy arrays: outer
        (steps taken), status (CONVERGED when the rule was met), objective and
        min_dist at the last step; solution() then gives the stopping step's
        solution of every scenario."""
        n = self.n_scen
        outer = np.zeros(n, dtype=np.int32)
        stat = np.zeros(n, dtype=np.int32)
        J = np.zeros(n, dtype=np.float64)
        D = np.zeros(n, dtype=np.float64)
        _check(lib().tadmm_sqp(self.h, float(tol), int(max_iter), int(max_outer), float(obj_rtol), float(dist_tol),
                               outer.ctypes.data_as(_i32p), stat.ctypes.data_as(_i32p),
                               J.ctypes.data_as(C.POINTER(C.c_double)), D.ctypes.data_as(C.POINTER(C.c_double)),
                               C.c_void_p(_stream_ptr(stream))), "tadmm_sqp")
        return dict(outer=outer, status=stat, objective=J, min_dist=D)

    def penalty(self):
        """Final rho per scenario and the number of residual-balancing changes."""
        rho = np.zeros(self.n_scen, dtype=np.float64)
        chg = np.zeros(self.n_scen, dtype=np.int32)
        _check(lib().tadmm_get_penalty(self.h, rho.ctypes.data_as(C.POINTER(C.c_double)),
                                       chg.ctypes.data_as(C.POINTER(C.c_int32))), "tadmm_get_penalty")
        return dict(rho=rho, changes=chg)

    def split(self, sol):
        """Splits packed host results into per-scenario arrays (X [N,T+1,nx], U, theta [P,T], W)."""
        b = self.batch
        out = []
        xo = uo = to = 0
        for k in range(self.n_scen):
            N, T, P = int(b.N[k]), int(b.T[k]), int(b.P[k])
            nX, nU, nT = N * (T + 1) * b.nx, N * T * b.nu, P * T
            out.append(dict(X=np.asarray(sol["X"][xo:xo + nX]).reshape(N, T + 1, b.nx),
                            U=np.asarray(sol["U"][uo:uo + nU]).reshape(N, T, b.nu),
                            W=np.asarray(sol["W"][uo:uo + nU]).reshape(N, T, b.nu),
                            theta=np.asarray(sol["theta"][to:to + nT]).reshape(P, T),
                            status=int(sol["status"][k]), iters=int(sol["iters"][k]),
                            r=float(sol["res"][k, 0]), s=float(sol["res"][k, 1])))
            xo += nX; uo += nU; to += nT
        return out


def version() -> str:
    return lib().tadmm_version().decode()


def solve(batch, tol: float = 1e-4, max_iter: int = 500, device: bool = False, **kw):
    """One-shot solve.  device=False: returns (per-scenario results as numpy
    arrays, solver).  device=True: returns (X, U, info, solver) with X and U
    float64 CUDA tensors in the packed layouts of tadmm_get_solution and info
    holding theta and W (CUDA tensors) and status, iters, res (numpy); the solver
    stays open for backward() and is closed by the caller."""
    s = Solver(batch, **kw)
    s.solve(tol, max_iter)
    if device:
        sol = s.solution(device=True)
        X, U = sol.pop("X"), sol.pop("U")
        return X, U, sol, s
    return s.split(s.solution()), s


class TADMMFunction:
    """Differentiable solve: X = TADMMFunction.apply(Qd, Rd, goal, solver, ...).

    Qd [sum N, nx] (diag Q per agent, with Qf = qf_tie * Q), Rd [sum N, nu] and
    goal [sum N, nx] (the goal state x_ref) are float64 torch tensors (CUDA or
    host).  The forward pass writes them into `solver`'s device data
    (tadmm_update_costs, no host round trip for CUDA tensors), solves to `tol`
    and returns the polished states at the final active set (packed layout of
    X, float64 on the GPU).  The backward pass runs the implicit-KKT adjoint
    kernel.
    """

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Qd, Rd, goal, solver, tol, max_iter, qf_tie, theta_eps):
                solver.update_costs(Qd=Qd, Rd=Rd, Qfd=qf_tie * Qd, x_ref=goal)
                solver.solve(tol, max_iter)
                X, st = solver.polished_states(theta_eps=theta_eps)
                ctx.solver, ctx.qf_tie, ctx.theta_eps = solver, qf_tie, theta_eps
                ctx.status = st
                return X if Qd.is_cuda else X.cpu()

            @staticmethod
            def backward(ctx, grad_X):
                g = ctx.solver.backward(grad_X.detach().to("cuda", dtype=torch.float64).contiguous(),
                                        theta_eps=ctx.theta_eps, polished=False)
                dev = grad_X.device
                gQ = torch.from_numpy(g["gQ"] + ctx.qf_tie * g["gQf"]).to(dev)
                return gQ, torch.from_numpy(g["gR"]).to(dev), torch.from_numpy(g["gGoal"]).to(dev), \
                    None, None, None, None, None

        return _F

    @classmethod
    def apply(cls, Qd, Rd, goal, solver, tol=1e-4, max_iter=500, qf_tie=10.0, theta_eps=1e-9):
        return cls._fn().apply(Qd, Rd, goal, solver, tol, max_iter, qf_tie, theta_eps)
