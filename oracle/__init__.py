"""ctypes binding of the plain-C FP64 oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package; the product library never does.  The C code lives in
`tadmm_oracle.c`; see its header for what each routine computes and which part
of the paper it follows.  Parity against numbers printed in the paper is
unpinned (the paper prints no worked example); the routines are pinned in the
tests against closed forms, bounded least squares, brute force and KKT
invariants.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional

import numpy as np

from . import build as _build

START_COLD, START_HOT, START_TURBO, START_HOMOTOPY = 0, 1, 2, 3
QP_COLD, QP_LQR, QP_GIVEN = 0, 1, 2
CONVERGED, NOT_CONVERGED, QP_FAIL, NUMERIC = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)
_i8p = C.POINTER(C.c_int8)
_u8p = C.POINTER(C.c_uint8)


class AgentQP(C.Structure):
    _fields_ = [("T", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("A", _dp), ("B", _dp),
                ("Hx", _dp), ("gx", _dp), ("Hu", _dp), ("x0", _dp), ("umin", _dp), ("umax", _dp)]


class Scenario(C.Structure):
    _fields_ = [("N", C.c_int), ("T", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("dp", C.c_int),
                ("A", _dp), ("B", _dp), ("Qd", _dp), ("Rd", _dp), ("Qfd", _dp),
                ("x_init", _dp), ("x_ref", _dp), ("umin", _dp), ("umax", _dp),
                ("a", _dp), ("w0", _dp), ("d_min", C.c_double), ("rho", C.c_double),
                ("P", C.c_int), ("pairs", C.POINTER(C.c_int)), ("Ai", _dp), ("Bi", _dp)]


class Options(C.Structure):
    _fields_ = [("start_mode", C.c_int), ("as_max", C.c_int), ("eps_rel", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("nthreads", C.c_int),
                ("adapt_every", C.c_int), ("adapt_mu", C.c_double), ("adapt_tau", C.c_double),
                ("relax_alpha", C.c_double), ("restart_eta", C.c_double)]


class Result(C.Structure):
    _fields_ = [("X", _dp), ("U", _dp), ("theta", _dp), ("W", _i8p), ("mu", _dp), ("trace", _dp),
                ("iters", C.c_int), ("status", C.c_int), ("r", C.c_double), ("s", C.c_double),
                ("as_iters", C.c_int64), ("inv_dev", C.c_double), ("rho_final", C.c_double),
                ("rho_changes", C.c_int), ("restarts", C.c_int), ("homotopy_steps", C.c_int64)]


class GlobalResult(C.Structure):
    _fields_ = [("X", _dp), ("U", _dp), ("mu_h", _dp), ("act_h", _u8p), ("W", _i8p), ("mu_u", _dp),
                ("iters", C.c_int), ("status", C.c_int), ("obj", C.c_double)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        _LIB = C.CDLL(path)
        _LIB.orc_agent_qp_solve.argtypes = [C.POINTER(AgentQP), C.c_int, C.c_int, C.c_double, _dp, _i8p,
                                            _dp, _dp, C.POINTER(C.c_int)]
        _LIB.orc_agent_eqp.argtypes = [C.POINTER(AgentQP), _i8p, _dp, _dp, _dp]
        _LIB.orc_agent_qp_homotopy.argtypes = [C.POINTER(AgentQP), _dp, C.c_int, C.c_double, _dp, _i8p, _dp, _dp,
                                               C.POINTER(C.c_int), C.POINTER(C.c_int)]
        _LIB.orc_agent_bruteforce.argtypes = [C.POINTER(AgentQP), C.c_double, _dp, _i8p]
        _LIB.orc_halfspace_project.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp, _dp, _dp]
        _LIB.orc_halfspace_project.restype = C.c_double
        _LIB.orc_agent_xupdate.argtypes = [C.POINTER(Scenario), C.c_int, _dp, C.c_int, C.c_int, C.c_double, _dp,
                                           _i8p, _dp, _dp, C.POINTER(C.c_int)]
        _LIB.orc_admm.argtypes = [C.POINTER(Scenario), C.POINTER(Options), C.POINTER(Result)]
        _LIB.orc_admm_batch.argtypes = [C.POINTER(Scenario), C.c_int, C.POINTER(Options),
                                        C.POINTER(Result), C.c_int]
        _LIB.orc_global_qp.argtypes = [C.POINTER(Scenario), C.c_int, C.c_double, C.POINTER(GlobalResult)]
        _LIB.orc_global_gradient.argtypes = [C.POINTER(Scenario), _u8p, _i8p, _dp, C.c_double, _dp, _dp,
                                             _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_int)]
    return _LIB


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- agent QP
class _AgentQPData:
    def __init__(self, A, B, Hx, gx, Hu, x0, umin, umax):
        self.arrs = [_f64(v) for v in (A, B, Hx, gx, Hu, x0, umin, umax)]
        A, B, Hx, gx, Hu, x0, umin, umax = self.arrs
        self.T, self.nx = Hx.shape
        self.nu = Hu.shape[0]
        self.s = AgentQP(self.T, self.nx, self.nu, _d(A), _d(B), _d(Hx), _d(gx), _d(Hu), _d(x0),
                         _d(umin), _d(umax))


def agent_qp_solve(A, B, Hx, gx, Hu, x0, umin, umax, start=QP_LQR, as_max=1000, eps_rel=1e-12,
                   u=None, W=None):
    """Per-agent box-constrained LQ problem (dense KKT active set)."""
    q = _AgentQPData(A, B, Hx, gx, Hu, x0, umin, umax)
    T, nx, nu = q.T, q.nx, q.nu
    u = np.zeros((T, nu)) if u is None else _f64(u).copy()
    W = np.zeros((T, nu), dtype=np.int8) if W is None else np.ascontiguousarray(W, dtype=np.int8).copy()
    x = np.zeros((T + 1, nx))
    mu = np.zeros((T, nu))
    n = C.c_int(0)
    st = lib().orc_agent_qp_solve(C.byref(q.s), start, as_max, eps_rel, _d(u), W.ctypes.data_as(_i8p),
                                  _d(x), _d(mu), C.byref(n))
    return dict(status=st, u=u, W=W, x=x, mu=mu, n_eqp=n.value)


def agent_qp_homotopy(A, B, Hx, gx_old, gx, Hu, x0, umin, umax, u, W, mu, as_max=1000, eps_rel=1e-12):
    """Homotopy hot start from the optimum (u, W, mu) for the state linear term
    gx_old to the QP with gx (qpOASES-style parametric active set)."""
    q = _AgentQPData(A, B, Hx, gx, Hu, x0, umin, umax)
    T, nx, nu = q.T, q.nx, q.nu
    g0 = _f64(gx_old).reshape(T, nx)
    u = _f64(u).copy()
    W = np.ascontiguousarray(W, dtype=np.int8).copy()
    mu = _f64(mu).copy()
    x = np.zeros((T + 1, nx))
    n, ns = C.c_int(0), C.c_int(0)
    st = lib().orc_agent_qp_homotopy(C.byref(q.s), _d(g0), as_max, eps_rel, _d(u), W.ctypes.data_as(_i8p),
                                     _d(x), _d(mu), C.byref(n), C.byref(ns))
    return dict(status=st, u=u, W=W, x=x, mu=mu, n_eqp=n.value, n_steps=ns.value)


def agent_eqp(A, B, Hx, gx, Hu, x0, umin, umax, W=None):
    q = _AgentQPData(A, B, Hx, gx, Hu, x0, umin, umax)
    T, nx, nu = q.T, q.nx, q.nu
    W = np.zeros((T, nu), dtype=np.int8) if W is None else np.ascontiguousarray(W, dtype=np.int8)
    u = np.zeros((T, nu)); x = np.zeros((T + 1, nx)); mu = np.zeros((T, nu))
    rc = lib().orc_agent_eqp(C.byref(q.s), W.ctypes.data_as(_i8p), _d(u), _d(x), _d(mu))
    if rc != 0:
        raise RuntimeError("singular KKT system")
    return dict(u=u, x=x, mu=mu)


def agent_bruteforce(A, B, Hx, gx, Hu, x0, umin, umax, tol=1e-9):
    q = _AgentQPData(A, B, Hx, gx, Hu, x0, umin, umax)
    u = np.zeros((q.T, q.nu)); W = np.zeros((q.T, q.nu), dtype=np.int8)
    found = lib().orc_agent_bruteforce(C.byref(q.s), tol, _d(u), W.ctypes.data_as(_i8p))
    return dict(found=found, u=u, W=W)


def halfspace_project(a, d, vi, vj):
    """Projection of (vi, vj) onto {a'(wi - wj) >= d}; returns (theta, wi, wj)."""
    a, vi, vj = _f64(a), _f64(vi), _f64(vj)
    wi = np.zeros_like(vi); wj = np.zeros_like(vj)
    th = lib().orc_halfspace_project(a.shape[0], _d(a), float(d), _d(vi), _d(vj), _d(wi), _d(wj))
    return th, wi, wj


# ---------------------------------------------------------------- scenarios
class _ScenarioData:
    """Keeps the numpy slices of scenario k of a Batch alive for the C call."""

    def __init__(self, batch, k: int):
        ao, po, so = batch.agent_off, batch.pairstep_off, batch.agentstep_off
        N, T = int(batch.N[k]), int(batch.T[k])
        sl = lambda arr, off: np.ascontiguousarray(arr[off[k]:off[k + 1]], dtype=np.float64)
        self.N, self.T, self.nx, self.nu, self.dp = N, T, batch.nx, batch.nu, batch.dp
        self.P = int(batch.P[k])
        self.keep = dict(A=_f64(batch.A), B=_f64(batch.B), Qd=sl(batch.Qd, ao), Rd=sl(batch.Rd, ao),
                         Qfd=sl(batch.Qfd, ao), x_init=sl(batch.x_init, ao), x_ref=sl(batch.x_ref, ao),
                         umin=_f64(batch.umin), umax=_f64(batch.umax), a=sl(batch.a, po),
                         w0=sl(batch.w0, so))
        if self.keep["a"].size == 0:
            self.keep["a"] = np.zeros(1)
        listed = getattr(batch, "pair_ij", None) is not None
        if listed:
            pl = np.ascontiguousarray(batch.pairs_of(k), dtype=np.int32).reshape(-1)
            self.keep["pairs"] = pl if pl.size else np.zeros(2, dtype=np.int32)
        hetero = getattr(batch, "A_agent", None) is not None
        if hetero:
            self.keep["Ai"] = sl(batch.A_agent.reshape(-1, batch.nx * batch.nx), ao)
            self.keep["Bi"] = sl(batch.B_agent.reshape(-1, batch.nx * batch.nu), ao)
        kp = self.keep
        self.s = Scenario(N, T, batch.nx, batch.nu, batch.dp, _d(kp["A"]), _d(kp["B"]), _d(kp["Qd"]),
                          _d(kp["Rd"]), _d(kp["Qfd"]), _d(kp["x_init"]), _d(kp["x_ref"]),
                          _d(kp["umin"]), _d(kp["umax"]), _d(kp["a"]), _d(kp["w0"]),
                          float(batch.d_min[k]), float(batch.rho[k]), self.P,
                          kp["pairs"].ctypes.data_as(C.POINTER(C.c_int)) if listed else None,
                          _d(kp["Ai"]) if hetero else None, _d(kp["Bi"]) if hetero else None)


class _ResultData:
    def __init__(self, sd: _ScenarioData, max_iter: int, trace: bool):
        N, T, nx, nu = sd.N, sd.T, sd.nx, sd.nu
        self.X = np.zeros((N, T + 1, nx))
        self.U = np.zeros((N, T, nu))
        self.theta = np.zeros((max(sd.P, 1), T))
        self.W = np.zeros((N, T, nu), dtype=np.int8)
        self.mu = np.zeros((N, T, nu))
        self.trace = np.zeros((max(max_iter, 1), 2)) if trace else None
        self.r = Result(_d(self.X), _d(self.U), _d(self.theta), self.W.ctypes.data_as(_i8p), _d(self.mu),
                        _d(self.trace) if trace else None, 0, 0, 0.0, 0.0, 0, 0.0, 0.0, 0)
        self.P = sd.P

    def to_dict(self):
        r = self.r
        out = dict(X=self.X, U=self.U, theta=self.theta[:self.P], W=self.W, mu=self.mu,
                   iters=r.iters, status=r.status, r=r.r, s=r.s, as_iters=int(r.as_iters),
                   inv_dev=r.inv_dev, rho_final=r.rho_final, rho_changes=r.rho_changes,
                    restarts=r.restarts, homotopy_steps=int(r.homotopy_steps))
        if self.trace is not None:
            out["trace"] = self.trace[:r.iters]
        return out


def _options(start_mode, as_max, eps_rel, tol, max_iter, nthreads, adapt=None, alpha=1.0, restart=0.0):
    ae, am, at = (0, 10.0, 2.0) if adapt is None else adapt
    return Options(start_mode, as_max, eps_rel, tol, max_iter, nthreads, ae, am, at, alpha, restart)


def agent_xupdate(batch, k: int, i: int, h, start=QP_LQR, as_max=None, eps_rel=1e-12):
    """First-principles x-update of agent i of scenario k for a coupling term h [T, dp]."""
    sd = _ScenarioData(batch, k)
    T, nx, nu = sd.T, sd.nx, sd.nu
    hh = _f64(h).reshape(T, sd.dp)
    u = np.zeros((T, nu)); W = np.zeros((T, nu), dtype=np.int8); x = np.zeros((T + 1, nx)); mu = np.zeros((T, nu))
    n = C.c_int(0)
    st = lib().orc_agent_xupdate(C.byref(sd.s), i, _d(hh), start, as_max or 10 * T * nu + 10, eps_rel, _d(u),
                                 W.ctypes.data_as(_i8p), _d(x), _d(mu), C.byref(n))
    return dict(status=st, u=u, W=W, x=x, mu=mu, n_eqp=n.value)


def admm(batch, k: int = 0, start_mode=START_TURBO, tol=1e-4, max_iter=500, as_max=None,
         eps_rel=1e-12, nthreads=0, trace=False, adapt=None, alpha=1.0, restart=0.0):
    """Literal vector-form ADMM on scenario k of `batch`; adapt = (every, mu, tau)
    turns on residual balancing of rho; alpha != 1 over-relaxes the projection
    and dual update (Boyd et al. 2011, Sec. 3.4.3)."""
    sd = _ScenarioData(batch, k)
    if as_max is None:
        as_max = 10 * sd.T * sd.nu + 10
    rd = _ResultData(sd, max_iter, trace)
    o = _options(start_mode, as_max, eps_rel, tol, max_iter, nthreads, adapt, alpha, restart)
    lib().orc_admm(C.byref(sd.s), C.byref(o), C.byref(rd.r))
    return rd.to_dict()


def admm_batch(batch, idx: Optional[List[int]] = None, start_mode=START_TURBO, tol=1e-4, max_iter=500,
               as_max=None, eps_rel=1e-12, nthreads=None, adapt=None, alpha=1.0, restart=0.0):
    """ADMM on several scenarios in parallel over host cores. Returns (results, threads used)."""
    idx = list(range(batch.n_scen)) if idx is None else list(idx)
    sds = [_ScenarioData(batch, k) for k in idx]
    rds = [_ResultData(sd, max_iter, False) for sd in sds]
    S = len(idx)
    sarr = (Scenario * S)(*[sd.s for sd in sds])
    rarr = (Result * S)(*[rd.r for rd in rds])
    am = as_max if as_max is not None else 10 * int(batch.T.max()) * batch.nu + 10
    o = _options(start_mode, am, eps_rel, tol, max_iter, 0, adapt, alpha, restart)
    nt = os.cpu_count() if nthreads is None else nthreads
    used = lib().orc_admm_batch(sarr, S, C.byref(o), rarr, nt)
    out = []
    for rd, rr in zip(rds, rarr):
        rd.r = rr
        out.append(rd.to_dict())
    return out, used


def global_qp(batch, k: int = 0, as_max=100000, eps_rel=1e-12):
    """Centralized linearized QP (Eq. 1 with halfspaces), condensed, active set."""
    sd = _ScenarioData(batch, k)
    N, T, nx, nu, P = sd.N, sd.T, sd.nx, sd.nu, sd.P
    X = np.zeros((N, T + 1, nx)); U = np.zeros((N, T, nu))
    mu_h = np.zeros((max(P, 1), T)); act = np.zeros((max(P, 1), T), dtype=np.uint8)
    W = np.zeros((N, T, nu), dtype=np.int8); mu_u = np.zeros((N, T, nu))
    r = GlobalResult(_d(X), _d(U), _d(mu_h), act.ctypes.data_as(_u8p), W.ctypes.data_as(_i8p), _d(mu_u),
                     0, 0, 0.0)
    rc = lib().orc_global_qp(C.byref(sd.s), as_max, eps_rel, C.byref(r))
    if rc != 0:
        raise RuntimeError("global QP build failed")
    return dict(X=X, U=U, mu_h=mu_h[:P], act_h=act[:P], W=W, mu_u=mu_u, iters=r.iters, status=r.status,
                obj=r.obj)


def global_gradient(batch, k: int, act_h, W, targets, qf_tie=10.0):
    """Polished solution at the active set and the implicit-KKT loss gradient.

    Also returns the polished point's multipliers (mu_h [P, T] of the
    halfspaces, mu_u [N, T, nu] of the held bounds) and the number of active
    halfspace rows found linearly dependent on the others."""
    sd = _ScenarioData(batch, k)
    N, T, nx, nu, P = sd.N, sd.T, sd.nx, sd.nu, sd.P
    act = np.zeros((max(P, 1), T), dtype=np.uint8)
    act[:P] = np.asarray(act_h, dtype=np.uint8).reshape(P, T)
    Wc = np.ascontiguousarray(W, dtype=np.int8).reshape(N, T, nu)
    tg = _f64(targets).reshape(N, T, sd.dp)
    X = np.zeros((N, T + 1, nx)); U = np.zeros((N, T, nu)); loss = np.zeros(1)
    gQ = np.zeros((N, nx)); gR = np.zeros((N, nu)); gG = np.zeros((N, nx))
    mu_h = np.zeros((max(P, 1), T)); mu_u = np.zeros((N, T, nu)); ndep = C.c_int(0)
    rc = lib().orc_global_gradient(C.byref(sd.s), act.ctypes.data_as(_u8p), Wc.ctypes.data_as(_i8p),
                                   _d(tg), qf_tie, _d(X), _d(U), _d(loss), _d(gQ), _d(gR), _d(gG),
                                   _d(mu_h), _d(mu_u), C.byref(ndep))
    if rc != 0:
        raise RuntimeError(f"gradient failed ({rc})")
    return dict(X=X, U=U, loss=float(loss[0]), gQ=gQ, gR=gR, gGoal=gG, mu_h=mu_h[:P], mu_u=mu_u,
                n_dependent=int(ndep.value))


def relinearize(batch, X_list):
    """One outer step of a linearize-and-solve loop over the collision
    constraint |p_i - p_j| >= d_min (its halfspace linearization, Sec. III):
    returns a copy of `batch` whose normals are a_ijt = (p_it - p_jt) /
    |p_it - p_jt| at the positions of X_list[k] ([N, T+1, nx] per scenario;
    unchanged where the positions coincide) and whose initial consensus
    positions w0 are those positions.  Plain numpy: |d|^2 summed component by
    component, then sqrt and division, each correctly rounded."""
    import dataclasses
    a = batch.a.copy()
    w0 = batch.w0.copy()
    po, so, dp = batch.pairstep_off, batch.agentstep_off, batch.dp
    for k in range(batch.n_scen):
        X = np.asarray(X_list[k], dtype=np.float64)
        N, T = int(batch.N[k]), int(batch.T[k])
        pos = X[:, 1:, :dp]                                  # [N, T, dp]
        w0[so[k]:so[k + 1]] = pos.reshape(N * T, dp)
        for pk, (i, j) in enumerate(batch.pairs_of(k)):
            d = pos[i] - pos[j]                              # [T, dp]
            n2 = d[:, 0] * d[:, 0]
            for c in range(1, dp):
                n2 = n2 + d[:, c] * d[:, c]
            ok = n2 > 0.0
            nr = np.sqrt(np.where(ok, n2, 1.0))
            rows = a[po[k] + pk * T: po[k] + (pk + 1) * T]
            rows[ok] = d[ok] / nr[ok, None]
    return dataclasses.replace(batch, a=a, w0=w0)


def objective(batch, k: int, X, U) -> float:
    """Objective of Eq. (1) for scenario k at states X [N, T+1, nx] and inputs
    U [N, T, nu]: every agent's sum over t < T of (x_t - x_ref)' Q (x_t - x_ref)
    + u_t' R u_t, plus (x_T - x_ref)' Q_T (x_T - x_ref).  The t = 0 term is kept
    (it is constant in the decision variables).  Plain numpy sums."""
    ao = batch.agent_off
    sl = slice(int(ao[k]), int(ao[k + 1]))
    X = np.asarray(X, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    e = X - batch.x_ref[sl][:, None, :]                          # [N, T+1, nx]
    stage = (e[:, :-1, :] ** 2 * batch.Qd[sl][:, None, :]).sum()
    inputs = (U ** 2 * batch.Rd[sl][:, None, :]).sum()
    final = (e[:, -1, :] ** 2 * batch.Qfd[sl]).sum()
    return float(stage + inputs + final)


def min_distance(batch, k: int, X) -> float:
    """Smallest Euclidean distance |p_it - p_jt| over the coupled pairs of
    scenario k and the constrained steps t = 1..T (inf without pairs)."""
    X = np.asarray(X, dtype=np.float64)
    pos = X[:, 1:, :batch.dp]
    best = np.inf
    for i, j in batch.pairs_of(k):
        d = pos[i] - pos[j]
        best = min(best, float(np.sqrt((d * d).sum(axis=1)).min()))
    return best


def sqp(batch, k: int = 0, tol=1e-4, max_iter=500, max_outer=10, obj_rtol=1e-4, dist_tol=None, **admm_kw):
    """Sequential linearize-and-solve loop over the collision constraint of
    Eq. (1) for scenario k: outer step m solves the halfspace-linearized QP by
    ADMM (`admm`, options passed through), then stops when the solve converged,
    m >= 2, the objective changed by at most obj_rtol relative to step m - 1
    and every pair is at least d_min - dist_tol apart at t = 1..T (the
    termination rule of Sec. V.A: relative objective change and collision-free
    at every step), else re-linearizes at the solution (`relinearize`) and
    repeats, for at most max_outer steps.  dist_tol None: 2 sqrt(dp) tol (a
    converged solve's positions are within tol of consensus copies that satisfy
    the halfspace exactly).  Returns the last step's ADMM result with `outer`
    (steps taken), `sqp_status` (0 stopped by the rule, 1 max_outer reached),
    `objective`, `min_dist` and `objectives` (one per step)."""
    if dist_tol is None:
        dist_tol = 2.0 * np.sqrt(batch.dp) * tol
    b = batch.subset([k])
    d_min = float(b.d_min[0])
    J_prev, Js = None, []
    for m in range(1, max_outer + 1):
        o = admm(b, 0, tol=tol, max_iter=max_iter, **admm_kw)
        J = objective(b, 0, o["X"], o["U"])
        D = min_distance(b, 0, o["X"])
        Js.append(J)
        done = (o["status"] == CONVERGED and J_prev is not None and abs(J - J_prev) <= obj_rtol * abs(J_prev)
                and D >= d_min - dist_tol)
        if done or m == max_outer:
            break
        b = relinearize(b, [o["X"]])
        J_prev = J
    return dict(o, outer=m, sqp_status=0 if done else 1, objective=J, min_dist=D, objectives=Js)
