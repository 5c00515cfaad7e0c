"""Pins of the CPU FP64 oracle against things other than itself.

Each test checks one oracle routine against an independent formulation:
condensed least squares, SciPy's bounded-variable least squares, exhaustive
enumeration, a numpy adjoint recursion (the costate identity of Sec. IV.B),
SLSQP for the consensus projection, the KKT conditions of the centralized QP
of Eq. (1), finite differences for the gradient and the problem-size table of
Sec. V.A (Table 1).
"""
import os

import dataclasses

import numpy as np
import pytest
from scipy.optimize import lsq_linear, minimize

import oracle
from instances import make_workload, random_scenario, pair_list
from instances.generator import SplitMix64, make_batch, build_scenario
from tests.helpers import agent_condensed_qp, condensed, costate_gradient, random_agent_qp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ sizes
def test_table1_problem_dimensions():
    """Sec. V.A Table 1: per-agent variables (T+1)nx + T nu, dynamics rows T nx,
    and about N(N-1)/2 collision rows per step.  The table prints "~" and counts
    T steps for 2 agents but T+1 for the others; the build constrains t = 1..T
    (x_0 is data), i.e. N(N-1)/2 * T rows."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_problem_dimensions.txt"))
    T, nx, nu = 20, 4, 2
    for N, nvar, ndyn, ncol in rows:
        N = int(N)
        assert N * ((T + 1) * nx + T * nu) == nvar
        assert N * T * nx == ndyn
        assert ncol in (N * (N - 1) // 2 * T, N * (N - 1) // 2 * (T + 1))
    b = make_workload("ring14")
    assert b.a.shape[0] == 91 * 20 and b.w0.shape[0] == 14 * 20
    assert b.N[0] == 14 and b.T[0] == 20


# ------------------------------------------------------------------ generator
def test_generator_deterministic_and_certified():
    b1 = make_workload("mixed", n_scen=6)
    b2 = make_workload("mixed", n_scen=6)
    for f in ("N", "T", "x_init", "x_ref", "a", "w0"):
        assert np.array_equal(getattr(b1, f), getattr(b2, f))
    # the first scenarios do not depend on the batch size
    b3 = make_workload("mixed", n_scen=3)
    assert np.array_equal(b3.a, b1.a[:b3.a.shape[0]])
    for k in range(b1.n_scen):
        s = b1.scenario(k)
        N, T, d = int(s.N[0]), int(s.T[0]), float(s.d_min[0])
        g = s.w0.reshape(N, T, 2)
        pl = pair_list(N)
        a = s.a.reshape(len(pl), T, 2)
        assert np.allclose(np.linalg.norm(a, axis=-1), 1.0)
        sep = np.einsum("ptc,ptc->pt", a, g[pl[:, 0]] - g[pl[:, 1]])
        assert sep.min() >= 1.1 * d - 1e-12          # the guess satisfies every halfspace
        st = s.x_init[:, :2]
        dd = np.linalg.norm(st[pl[:, 0]] - st[pl[:, 1]], axis=-1)
        assert dd.min() >= 2 * d                      # rejection-sampled starts
        # guesses are the zero-input trajectories of the double integrator
        for i in range(N):
            x = s.x_init[i].copy()
            for t in range(T):
                x = s.A @ x
                assert np.allclose(x[:2], g[i, t], atol=1e-12)


def test_splitmix64_reference_values():
    """SplitMix64 (Steele, Lea & Flood 2014) outputs for seed 0: the published
    first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4."""
    r = SplitMix64(0)
    v = r.next_u64(2)
    assert int(v[0]) == 0xE220A8397B1DCDAF
    assert int(v[1]) == 0x6E789E6AA1B965F4


# ------------------------------------------------------------------ per-agent QP
@pytest.mark.parametrize("seed", range(6))
def test_eqp_unconstrained_equals_condensed_solve(seed):
    """Empty working set: the dense KKT solve equals the minimiser of the
    condensed quadratic (plain linear solve of its normal equations)."""
    rng = np.random.default_rng(seed)
    T = 5 + seed
    A, B, Hx, gx, Hu, x0, umin, umax = random_agent_qp(rng, T, double_integrator=seed % 2 == 0)
    out = oracle.agent_eqp(A, B, Hx, gx, Hu, x0, umin, umax)
    H, g, F, G = agent_condensed_qp(A, B, Hx, gx, Hu, x0)
    u = np.linalg.solve(H, -g)
    assert np.allclose(out["u"].ravel(), u, rtol=1e-10, atol=1e-10 * max(1, np.abs(u).max()))
    # forward pass satisfies the dynamics exactly (to rounding), Sec. IV.B
    x = out["x"]
    for t in range(T):
        assert np.allclose(x[t + 1], A @ x[t] + B @ out["u"][t], atol=1e-10 * max(1, np.abs(x).max()))
    # costate identity: gradient of the objective w.r.t. free inputs vanishes
    grad = costate_gradient(A, B, Hx, gx, Hu, x, out["u"])
    assert np.abs(grad).max() <= 1e-8 * max(1.0, np.abs(gx).max())


def _bvls(A, B, Hx, gx, Hu, x0, umin, umax):
    H, g, _, _ = agent_condensed_qp(A, B, Hx, gx, Hu, x0)
    L = np.linalg.cholesky(H)
    M = L.T
    rhs = -np.linalg.solve(L, g)
    T, nu = Hx.shape[0], B.shape[1]
    lb = np.tile(umin, T)
    ub = np.tile(umax, T)
    res = lsq_linear(M, rhs, bounds=(lb, ub), method="bvls", tol=1e-15, lsmr_tol=None)
    return res.x.reshape(T, nu), H, g


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("start", [oracle.QP_COLD, oracle.QP_LQR])
def test_box_qp_matches_bvls(seed, start):
    """Box-constrained per-agent QP: active-set result equals SciPy's BVLS on the
    equivalent bounded least-squares problem; KKT conditions hold."""
    rng = np.random.default_rng(100 + seed)
    T = 6 + 2 * seed
    A, B, Hx, gx, Hu, x0, umin, umax = random_agent_qp(rng, T, double_integrator=seed % 3 != 0)
    out = oracle.agent_qp_solve(A, B, Hx, gx, Hu, x0, umin, umax, start=start)
    assert out["status"] == oracle.CONVERGED
    u_ref, H, g = _bvls(A, B, Hx, gx, Hu, x0, umin, umax)
    scale = max(1.0, np.abs(u_ref).max())
    assert np.abs(out["u"] - u_ref).max() <= 1e-8 * scale
    # KKT: reduced gradient by the adjoint recursion
    grad = costate_gradient(A, B, Hx, gx, Hu, out["x"], out["u"])
    W = out["W"]
    gs = max(1.0, np.abs(grad).max())
    assert np.abs(grad[W == 0]).max(initial=0) <= 1e-8 * gs
    mu_ref = np.where(W == 1, grad, np.where(W == 2, -grad, 0.0))
    assert np.allclose(out["mu"], mu_ref, atol=1e-8 * gs)
    assert out["mu"].min() >= -1e-9 * gs
    lo = np.broadcast_to(umin, out["u"].shape)
    hi = np.broadcast_to(umax, out["u"].shape)
    assert np.all(out["u"] >= lo) and np.all(out["u"] <= hi)
    assert np.array_equal(out["u"][W == 1], lo[W == 1]) and np.array_equal(out["u"][W == 2], hi[W == 2])


@pytest.mark.parametrize("seed", range(10))
def test_box_qp_matches_bruteforce(seed):
    """Tiny QPs (T=3, nu=2: 3^6 working sets): exactly one KKT point exists and
    every start of the active-set method reaches it with the same active set."""
    rng = np.random.default_rng(200 + seed)
    A, B, Hx, gx, Hu, x0, umin, umax = random_agent_qp(rng, 3, box=0.3)
    bf = oracle.agent_bruteforce(A, B, Hx, gx, Hu, x0, umin, umax, tol=1e-10)
    assert bf["found"] == 1
    for start in (oracle.QP_COLD, oracle.QP_LQR):
        out = oracle.agent_qp_solve(A, B, Hx, gx, Hu, x0, umin, umax, start=start)
        assert out["status"] == oracle.CONVERGED
        assert np.allclose(out["u"], bf["u"], atol=1e-10)
        assert np.array_equal(out["W"], bf["W"])
    u_ref, _, _ = _bvls(A, B, Hx, gx, Hu, x0, umin, umax)
    assert np.allclose(bf["u"], u_ref, atol=1e-8)


def test_box_qp_hot_start_from_solution_is_one_solve():
    """Hot start from the optimal (u, W) of the same QP needs one EQP solve."""
    rng = np.random.default_rng(7)
    A, B, Hx, gx, Hu, x0, umin, umax = random_agent_qp(rng, 12)
    first = oracle.agent_qp_solve(A, B, Hx, gx, Hu, x0, umin, umax, start=oracle.QP_COLD)
    hot = oracle.agent_qp_solve(A, B, Hx, gx, Hu, x0, umin, umax, start=oracle.QP_GIVEN,
                                u=first["u"], W=first["W"])
    assert hot["n_eqp"] == 1
    assert np.allclose(hot["u"], first["u"], atol=1e-12)


def test_box_qp_wide_box_is_lqr():
    """umin = -inf-like, umax = +inf-like: the QP is the unconstrained LQR."""
    rng = np.random.default_rng(11)
    A, B, Hx, gx, Hu, x0, umin, umax = random_agent_qp(rng, 9)
    big = np.full_like(umin, 1e9)
    out = oracle.agent_qp_solve(A, B, Hx, gx, Hu, x0, -big, big, start=oracle.QP_LQR)
    assert out["n_eqp"] == 0 and not out["W"].any()
    H, g, _, _ = agent_condensed_qp(A, B, Hx, gx, Hu, x0)
    assert np.allclose(out["u"].ravel(), np.linalg.solve(H, -g), atol=1e-9)


def test_as_max_reports_qp_fail():
    rng = np.random.default_rng(3)
    A, B, Hx, gx, Hu, x0, umin, umax = random_agent_qp(rng, 10, box=0.2)
    out = oracle.agent_qp_solve(A, B, Hx, gx, Hu, x0, umin, umax, start=oracle.QP_COLD, as_max=1)
    assert out["status"] == oracle.QP_FAIL


# ------------------------------------------------------------------ consensus projection
@pytest.mark.parametrize("seed", range(6))
def test_halfspace_projection_matches_slsqp(seed):
    """The consensus step equals the Euclidean projection computed by a generic
    constrained solver, for active and inactive cases, 2D and 3D."""
    rng = np.random.default_rng(300 + seed)
    dp = 2 + seed % 2
    a = rng.standard_normal(dp)
    a /= np.linalg.norm(a)
    vi, vj = rng.standard_normal(dp), rng.standard_normal(dp)
    d = float(a @ (vi - vj)) + (0.7 if seed % 3 else -0.5)  # active unless seed % 3 == 0
    th, wi, wj = oracle.halfspace_project(a, d, vi, vj)
    v = np.concatenate([vi, vj])
    n = np.concatenate([a, -a])
    sol = minimize(lambda w: 0.5 * np.sum((w - v) ** 2), v, jac=lambda w: w - v, method="SLSQP",
                   constraints=[dict(type="ineq", fun=lambda w: n @ w - d, jac=lambda w: n)],
                   options=dict(ftol=1e-15, maxiter=200))
    assert np.allclose(np.concatenate([wi, wj]), sol.x, atol=1e-7)
    assert th >= 0.0
    assert float(a @ (wi - wj)) >= d - 1e-12
    assert np.allclose(wi - vi, th * a) and np.allclose(wj - vj, -th * a)
    if seed % 3 == 0:
        assert th == 0.0


# ------------------------------------------------------------------ ADMM
def test_admm_single_agent_one_iteration():
    """N = 1: no coupling; ADMM stops after one x-update at the box-QP solution."""
    b = random_scenario(seed=1, N=1, T=15)
    r = oracle.admm(b, 0, max_iter=50)
    assert r["status"] == oracle.CONVERGED and r["iters"] == 1
    Hx = np.tile(2 * b.Qd[0], (15, 1))
    Hx[-1] = 2 * b.Qfd[0]
    gx = -Hx * b.x_ref[0]
    u_ref, _, _ = _bvls(b.A, b.B, Hx, gx, 2 * b.Rd[0], b.x_init[0], b.umin, b.umax)
    assert np.abs(r["U"][0] - u_ref).max() <= 1e-8


def test_admm_start_modes_give_same_iterates():
    """Cold, hot and turbo starts only change the active-set path: every ADMM
    iterate is the unique per-agent QP solution, so the runs agree."""
    b = make_workload("pair")
    outs = [oracle.admm(b, 0, start_mode=m, max_iter=4, tol=0.0) for m in
            (oracle.START_COLD, oracle.START_HOT, oracle.START_TURBO)]
    for o in outs[1:]:
        assert np.abs(o["X"] - outs[0]["X"]).max() <= 1e-9
        assert np.abs(o["theta"] - outs[0]["theta"]).max() <= 1e-9
    assert outs[0]["as_iters"] >= outs[1]["as_iters"]


def test_admm_dual_invariant_and_uncoupled_case():
    """Two agents that never come close: every halfspace stays inactive, theta = 0,
    and the result equals two independent box-QP solutions."""
    T = 12
    starts = np.array([[-4.0, 0.0], [4.0, 0.0]])
    goals = np.array([[-4.0, 2.0], [4.0, -2.0]])
    x_init, x_ref, a, w0, c = build_scenario(starts, goals, T, 0.1, 0.5)
    b = make_batch([dict(N=2, T=T, x_init=x_init, x_ref=x_ref, a=a, w0=w0, d=0.5, rho=1.0, umax=1.0, c=c)],
                   dp=2, dt=0.1, umax=1.0)
    r = oracle.admm(b, 0, tol=1e-11, max_iter=3000)
    assert r["status"] == oracle.CONVERGED
    assert np.all(r["theta"] == 0.0)
    assert r["inv_dev"] <= 1e-12
    for i in range(2):
        Hx = np.tile(2 * b.Qd[i], (T, 1))
        Hx[-1] = 2 * b.Qfd[i]
        gx = -Hx * b.x_ref[i]
        u_ref, _, _ = _bvls(b.A, b.B, Hx, gx, 2 * b.Rd[i], b.x_init[i], b.umin, b.umax)
        assert np.abs(r["U"][i] - u_ref).max() <= 1e-7


def _global_kkt_check(b, g, tol):
    """KKT conditions of Eq. (1) with linearized halfspaces, written independently:
    stationarity H U + g = sum mu_h n_h + bound terms, feasibility, complementarity."""
    N, T, nx, nu, dp = int(b.N[0]), int(b.T[0]), b.nx, b.nu, b.dp
    pl = pair_list(N)
    m = T * nu
    Hs, gs, Fs, Gs = [], [], [], []
    for i in range(N):
        Hx = np.tile(2 * b.Qd[i], (T, 1))
        Hx[-1] = 2 * b.Qfd[i]
        Ai = b.A if b.A_agent is None else b.A_agent[i]
        Bi = b.B if b.B_agent is None else b.B_agent[i]
        H, gg, F, G = agent_condensed_qp(Ai, Bi, Hx, -Hx * b.x_ref[i], 2 * b.Rd[i], b.x_init[i])
        Hs.append(H); gs.append(gg); Fs.append(F); Gs.append(G)
    U = g["U"].reshape(N, m)
    grad = np.stack([Hs[i] @ U[i] + gs[i] for i in range(N)])
    a = b.a.reshape(len(pl), T, dp)
    res = grad.copy()
    worst_slack = np.inf
    for k, (i, j) in enumerate(pl):
        for t in range(1, T + 1):
            ni = a[k, t - 1] @ Gs[i][t][:dp]
            nj = -a[k, t - 1] @ Gs[j][t][:dp]
            slack = a[k, t - 1] @ ((Fs[i][t] + Gs[i][t] @ U[i])[:dp] - (Fs[j][t] + Gs[j][t] @ U[j])[:dp]) - b.d_min[0]
            worst_slack = min(worst_slack, slack)
            mu = g["mu_h"][k, t - 1]
            assert mu >= -tol
            assert abs(mu * slack) <= tol * max(1.0, abs(mu))
            res[i] -= mu * ni
            res[j] -= mu * nj
    Wf = g["W"].reshape(N, m)
    mu_u = g["mu_u"].reshape(N, m)
    res -= np.where(Wf == 1, mu_u, 0.0) - np.where(Wf == 2, mu_u, 0.0)
    assert worst_slack >= -tol
    assert np.abs(res).max() <= tol * max(1.0, np.abs(grad).max())
    assert mu_u.min() >= -tol


@pytest.mark.parametrize("seed,N,T", [(1, 3, 8), (2, 4, 6), (5, 3, 10)])
def test_global_qp_satisfies_kkt(seed, N, T):
    b = random_scenario(seed=seed, N=N, T=T, box=2.0)
    g = oracle.global_qp(b, 0)
    assert g["status"] == oracle.CONVERGED
    _global_kkt_check(b, g, 1e-8)


def test_admm_converges_to_global_qp():
    """The ADMM fixed point is the centralized optimum: run to tol 1e-10 and compare
    with the global QP; the halfspace multipliers are rho * theta."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=20.0)
    g = oracle.global_qp(b, 0)
    assert g["status"] == oracle.CONVERGED and g["act_h"].sum() > 0
    r = oracle.admm(b, 0, tol=1e-10, max_iter=20000)
    assert r["status"] == oracle.CONVERGED
    assert np.abs(r["X"] - g["X"]).max() <= 1e-7
    assert np.abs(b.rho[0] * r["theta"] - g["mu_h"]).max() <= 1e-5 * max(1, g["mu_h"].max())
    assert np.array_equal(r["W"], g["W"])
    assert r["inv_dev"] <= 1e-10


def test_residual_balancing_keeps_the_fixed_point():
    """Residual balancing of rho (Boyd et al. 2011, Sec. 3.4.1; an extension,
    off by default) changes the path, not the answer: started at a rho far
    from balanced, rho is changed several times and the run still converges to
    the global QP optimum, with the halfspace multipliers equal to
    rho_final * theta and the scaled-dual identity y = -theta a intact."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=0.5)
    g = oracle.global_qp(b, 0)
    assert g["status"] == oracle.CONVERGED and g["act_h"].sum() > 0
    r = oracle.admm(b, 0, tol=1e-10, max_iter=20000, adapt=(5, 10.0, 2.0))
    assert r["status"] == oracle.CONVERGED
    assert r["rho_changes"] >= 2
    assert np.abs(r["X"] - g["X"]).max() <= 1e-7
    assert np.abs(r["rho_final"] * r["theta"] - g["mu_h"]).max() <= 1e-5 * max(1, g["mu_h"].max())
    assert np.array_equal(r["W"], g["W"])
    assert r["inv_dev"] <= 1e-10
    # rho_final is rho times tau to the net number of raises
    k = np.log(r["rho_final"] / b.rho[0]) / np.log(2.0)
    assert abs(k - round(k)) < 1e-12 and abs(round(k)) <= r["rho_changes"]


def test_residual_balancing_never_due_is_plain_admm():
    """With the first balancing point past max_iter the run is the plain one, bit for bit."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=0.5)
    r0 = oracle.admm(b, 0, tol=0.0, max_iter=30)
    r1 = oracle.admm(b, 0, tol=0.0, max_iter=30, adapt=(31, 10.0, 2.0))
    assert r1["rho_changes"] == 0 and r1["rho_final"] == b.rho[0]
    assert np.array_equal(r0["X"], r1["X"]) and np.array_equal(r0["theta"], r1["theta"])


def test_heterogeneous_agents_equal_models_are_the_shared_run():
    """Per-agent dynamics that all equal the shared model reproduce the shared
    run bit for bit (ADMM iterates and the global QP)."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=0.5)
    na = int(b.N.sum())
    bh = dataclasses.replace(b, A_agent=np.tile(b.A, (na, 1, 1)), B_agent=np.tile(b.B, (na, 1, 1)))
    r0 = oracle.admm(b, 0, tol=0.0, max_iter=30)
    r1 = oracle.admm(bh, 0, tol=0.0, max_iter=30)
    assert np.array_equal(r0["X"], r1["X"]) and np.array_equal(r0["theta"], r1["theta"])
    g0, g1 = oracle.global_qp(b, 0), oracle.global_qp(bh, 0)
    assert np.array_equal(g0["X"], g1["X"]) and np.array_equal(g0["mu_h"], g1["mu_h"])


@pytest.mark.parametrize("seed,N,T", [(3, 3, 8), (5, 4, 10)])
def test_heterogeneous_agents_global_qp_and_admm_fixed_point(seed, N, T):
    """Mixed models (per-agent damping and mass): the oracle's condensed global
    QP satisfies the KKT conditions written with each agent's own A_i, B_i
    (numpy condensing), and its ADMM converges to that optimum."""
    from instances import heterogeneous_agents
    b = heterogeneous_agents(random_scenario(seed=seed, N=N, T=T, box=1.5, rho=20.0), seed=seed)
    assert not np.allclose(b.A_agent[0], b.A_agent[1])
    g = oracle.global_qp(b, 0)
    assert g["status"] == oracle.CONVERGED and g["act_h"].sum() > 0
    _global_kkt_check(b, g, 1e-8)
    r = oracle.admm(b, 0, tol=1e-10, max_iter=40000)
    assert r["status"] == oracle.CONVERGED
    assert np.abs(r["X"] - g["X"]).max() <= 1e-7
    assert np.abs(b.rho[0] * r["theta"] - g["mu_h"]).max() <= 1e-5 * max(1, g["mu_h"].max())
    assert np.array_equal(r["W"], g["W"])
    # the shared-model run is a different problem
    g0 = oracle.global_qp(dataclasses.replace(b, A_agent=None, B_agent=None), 0)
    assert np.abs(g0["X"] - g["X"]).max() > 1e-3


def test_over_relaxation_alpha_one_is_plain_admm():
    """alpha = 1 is no relaxation, bit for bit."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=0.5)
    r0 = oracle.admm(b, 0, tol=0.0, max_iter=30)
    r1 = oracle.admm(b, 0, tol=0.0, max_iter=30, alpha=1.0)
    assert np.array_equal(r0["X"], r1["X"]) and np.array_equal(r0["theta"], r1["theta"])


@pytest.mark.parametrize("alpha", [0.7, 1.6])
def test_over_relaxation_keeps_the_fixed_point(alpha):
    """Over-relaxed ADMM (Boyd et al. 2011, Sec. 3.4.3; an extension, off by
    default) has the same fixed point: it converges to the global QP optimum,
    with the halfspace multipliers rho * theta and y = -theta a intact."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=20.0)
    g = oracle.global_qp(b, 0)
    assert g["status"] == oracle.CONVERGED and g["act_h"].sum() > 0
    r = oracle.admm(b, 0, tol=1e-10, max_iter=40000, alpha=alpha)
    assert r["status"] == oracle.CONVERGED
    assert np.abs(r["X"] - g["X"]).max() <= 1e-7
    assert np.abs(b.rho[0] * r["theta"] - g["mu_h"]).max() <= 1e-5 * max(1, g["mu_h"].max())
    assert np.array_equal(r["W"], g["W"])
    assert r["inv_dev"] <= 1e-10


def test_accelerated_admm_keeps_the_fixed_point():
    """Accelerated ADMM with restart (Goldstein et al. 2014, combined residual in
    the max norm; evaluated on the oracle only) reaches the same global QP
    optimum, here in far fewer iterations; eta = 0 is the plain run."""
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=20.0)
    g = oracle.global_qp(b, 0)
    r0 = oracle.admm(b, 0, tol=1e-10, max_iter=40000)
    r = oracle.admm(b, 0, tol=1e-10, max_iter=40000, restart=0.999)
    assert r0["status"] == r["status"] == oracle.CONVERGED
    assert r["restarts"] > 0 and r["iters"] < r0["iters"] // 3
    assert np.abs(r["X"] - g["X"]).max() <= 1e-7
    assert np.abs(b.rho[0] * r["theta"] - g["mu_h"]).max() <= 1e-5 * max(1, g["mu_h"].max())
    assert np.array_equal(r["W"], g["W"])
    assert r["inv_dev"] <= 1e-10
    p0 = oracle.admm(b, 0, tol=0.0, max_iter=20)
    p1 = oracle.admm(b, 0, tol=0.0, max_iter=20, restart=0.0)
    assert np.array_equal(p0["X"], p1["X"]) and np.array_equal(p0["theta"], p1["theta"])


def test_over_relaxation_theta_form_equals_vector_form():
    """The pair-scalar form of over-relaxed ADMM that the GPU path runs, written
    here with numpy around the oracle's own x-update: with y_i = -theta a and the
    consensus copies w_i = s_i + phi a, w_j = s_j - phi a (s per agent and step,
    phi per pair and step), one iteration is
        theta' = max(0, theta + (d - alpha a.(p_i - p_j) - (1 - alpha)(a.(s_i - s_j) + 2 phi)) / 2)
        phi'   = (1 - alpha) phi + theta' - theta,   s' = alpha p + (1 - alpha) s
        h_i    = n_c s_i' + sum_j sigma_ij (phi' + theta') a_ij.
    Its iterates must equal the literal vector-form ADMM (per-side copies and
    scaled duals) to rounding."""
    alpha = 1.6
    b = random_scenario(seed=3, N=3, T=8, box=1.5, rho=1.0)
    N, T, dp = int(b.N[0]), int(b.T[0]), b.dp
    pl = pair_list(N)
    P = len(pl)
    a = b.a.reshape(P, T, dp)
    d = float(b.d_min[0])
    s = b.w0.reshape(N, T, dp).copy()
    phi = np.zeros((P, T))
    th = np.zeros((P, T))
    K = 25
    for k in range(K):
        h = (N - 1) * s.copy()
        for q, (i, j) in enumerate(pl):
            h[i] += (phi[q] + th[q])[:, None] * a[q]
            h[j] -= (phi[q] + th[q])[:, None] * a[q]
        X = np.stack([oracle.agent_xupdate(b, 0, i, h[i], start=oracle.QP_LQR)["x"] for i in range(N)])
        p = X[:, 1:, :dp]
        for q, (i, j) in enumerate(pl):
            ahat = alpha * np.einsum("tc,tc->t", a[q], p[i] - p[j]) \
                + (1 - alpha) * (np.einsum("tc,tc->t", a[q], s[i] - s[j]) + 2 * phi[q])
            tn = np.maximum(0.0, th[q] + (d - ahat) / 2)
            phi[q] = (1 - alpha) * phi[q] + tn - th[q]
            th[q] = tn
        s = alpha * p + (1 - alpha) * s
    r = oracle.admm(b, 0, tol=0.0, max_iter=K, alpha=alpha)
    assert r["iters"] == K
    assert np.abs(r["X"] - X).max() <= 1e-10 * max(1.0, np.abs(X).max())
    assert np.abs(r["theta"] - th).max() <= 1e-10 * max(1.0, np.abs(th).max())
    assert th.max() > 0  # halfspaces active: the test exercises the projection


def test_relinearization_at_the_guess_reproduces_the_normals():
    """Re-linearizing at the guess lines (the zero-input trajectories the
    instances are built from) gives back the instance's own halfspace normals
    and consensus guess: unit normals pointing from p_j to p_i, with
    a . (p_i - p_j) = |p_i - p_j|."""
    b = make_workload("mixed", n_scen=3)
    X_list = []
    for k in range(b.n_scen):
        sc = b.scenario(k)
        N, T = int(sc.N[0]), int(sc.T[0])
        X = np.zeros((N, T + 1, b.nx))
        X[:, 1:, :b.dp] = sc.w0.reshape(N, T, b.dp)
        X_list.append(X)
    r = oracle.relinearize(b, X_list)
    assert np.abs(r.a - b.a).max() <= 1e-15
    assert np.array_equal(r.w0, b.w0)
    assert np.abs(np.linalg.norm(r.a, axis=1) - 1.0).max() <= 1e-15
    k = 2
    sc = b.scenario(k)
    N, T = int(sc.N[0]), int(sc.T[0])
    pos = sc.w0.reshape(N, T, b.dp)
    a = r.scenario(k).a.reshape(-1, T, b.dp)
    d = pos[0] - pos[1]
    assert np.abs((a[0] * d).sum(-1) - np.linalg.norm(d, axis=-1)).max() <= 1e-14


def test_pair_list_of_all_pairs_is_the_dense_run():
    """Listing every pair explicitly (lexicographic) is the dense all-pairs run, bit for bit."""
    from instances import pair_list
    b = make_workload("mixed", n_scen=2)
    r0 = [oracle.admm(b, k, tol=0.0, max_iter=6) for k in range(2)]
    bl = dataclasses.replace(b, pair_count=b.P.astype(np.int32),
                             pair_ij=np.concatenate([pair_list(int(n)) for n in b.N]))
    for k in range(2):
        r1 = oracle.admm(bl, k, tol=0.0, max_iter=6)
        assert np.array_equal(r0[k]["X"], r1["X"]) and np.array_equal(r0[k]["theta"], r1["theta"])


def test_sparse_coupling_converges_to_its_global_qp():
    """Coupling only each agent's nearest neighbours: the ADMM fixed point is the
    centralized optimum of the QP with just those halfspaces, each agent's
    copy count n_c being its number of pairs (a wrong count moves the fixed
    point); the halfspace multipliers are rho * theta."""
    from instances import nearest_neighbour_pairs
    b = nearest_neighbour_pairs(random_scenario(seed=10, N=5, T=8, box=1.5, rho=20.0), 2)
    assert 0 < int(b.P[0]) < 10
    g = oracle.global_qp(b, 0)
    assert g["status"] == oracle.CONVERGED and g["act_h"].sum() > 0
    r = oracle.admm(b, 0, tol=1e-10, max_iter=40000)
    assert r["status"] == oracle.CONVERGED
    assert np.abs(r["X"] - g["X"]).max() <= 1e-7
    assert np.abs(b.rho[0] * r["theta"] - g["mu_h"]).max() <= 1e-5 * max(1, g["mu_h"].max())


def test_literal_reading_is_infeasible_and_does_not_converge():
    """Zero initial velocity with c = 1 guess lines (the literal reading): the
    agents cannot swap sides in 2 s, the halfspace QP is infeasible and the
    residual stalls."""
    b = make_workload("pair", literal=True)
    r = oracle.admm(b, 0, max_iter=300)
    assert r["status"] == oracle.NOT_CONVERGED and r["iters"] == 300
    assert r["r"] > 1e-2


# ------------------------------------------------------------------ gradient
def _loss(X, targets, dp):
    N, T1, _ = X.shape
    return float(((X[:, 1:, :dp] - targets.reshape(N, T1 - 1, dp)) ** 2).sum())


@pytest.mark.parametrize("seed,hetero", [(1, False), (4, False), (3, True)])
def test_gradient_matches_central_differences(seed, hetero):
    """Implicit-KKT gradient at the final active set equals central finite
    differences (h = 1e-6) of the re-solved centralized QP (also with per-agent
    dynamics)."""
    b = random_scenario(seed=seed, N=3, T=6, box=1.5)
    if hetero:
        from instances import heterogeneous_agents
        b = heterogeneous_agents(b, seed=seed)
    rng = np.random.default_rng(seed)
    targets = rng.uniform(-2, 2, size=(3 * 6, 2))
    g = oracle.global_qp(b, 0)
    gr = oracle.global_gradient(b, 0, g["act_h"], g["W"], targets, qf_tie=10.0)
    assert np.abs(gr["X"] - g["X"]).max() <= 1e-9
    h = 1e-6

    def solve_loss(mod):
        bb = b.subset([0])
        mod(bb)
        gg = oracle.global_qp(bb, 0)
        same = np.array_equal(gg["act_h"], g["act_h"]) and np.array_equal(gg["W"], g["W"])
        return _loss(gg["X"], targets, 2), same

    checked = 0
    for i in range(3):
        for r in range(4):
            def mq(bb, s):
                bb.Qd = bb.Qd.copy(); bb.Qfd = bb.Qfd.copy()
                bb.Qd[i, r] += s; bb.Qfd[i, r] += 10 * s
            lp, s1 = solve_loss(lambda bb: mq(bb, h))
            lm, s2 = solve_loss(lambda bb: mq(bb, -h))
            if s1 and s2:
                fd = (lp - lm) / (2 * h)
                assert abs(fd - gr["gQ"][i, r]) <= 1e-5 * max(1.0, abs(fd)), (i, r)
                checked += 1

            def mg(bb, s):
                bb.x_ref = bb.x_ref.copy(); bb.x_ref[i, r] += s
            lp, s1 = solve_loss(lambda bb: mg(bb, h))
            lm, s2 = solve_loss(lambda bb: mg(bb, -h))
            if s1 and s2:
                fd = (lp - lm) / (2 * h)
                assert abs(fd - gr["gGoal"][i, r]) <= 1e-5 * max(1.0, abs(fd)), (i, r)
                checked += 1
        for c in range(2):
            def mr(bb, s):
                bb.Rd = bb.Rd.copy(); bb.Rd[i, c] += s
            lp, s1 = solve_loss(lambda bb: mr(bb, h))
            lm, s2 = solve_loss(lambda bb: mr(bb, -h))
            if s1 and s2:
                fd = (lp - lm) / (2 * h)
                assert abs(fd - gr["gR"][i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, c)
                checked += 1
    assert checked >= 20


@pytest.mark.parametrize("seed", range(6))
def test_homotopy_hot_start_reaches_the_new_optimum(seed):
    """Parametric (homotopy) hot start, qpOASES-style (evaluated on the oracle
    only): from the optimum of a box QP, following the linear term to a new one
    ends at the new QP's optimum (SciPy BVLS), with at least one direction solve
    per working-set change and none left for the confirming active-set pass
    beyond one solve."""
    rng = np.random.default_rng(300 + seed)
    T = 8 + seed
    A, B, Hx, gx0, Hu, x0, umin, umax = random_agent_qp(rng, T, box=0.4)
    first = oracle.agent_qp_solve(A, B, Hx, gx0, Hu, x0, umin, umax, start=oracle.QP_COLD)
    assert first["status"] == oracle.CONVERGED
    gx1 = gx0 + rng.normal(0, 2.0, gx0.shape)
    h = oracle.agent_qp_homotopy(A, B, Hx, gx0, gx1, Hu, x0, umin, umax, first["u"], first["W"], first["mu"])
    assert h["status"] == oracle.CONVERGED
    u_ref, _, _ = _bvls(A, B, Hx, gx1, Hu, x0, umin, umax)
    assert np.abs(h["u"] - u_ref).max() <= 1e-8 * max(1.0, np.abs(u_ref).max())
    changes = int((h["W"] != first["W"]).sum())
    assert h["n_steps"] >= 1 and h["n_steps"] >= changes // 2
    assert h["n_eqp"] - h["n_steps"] == 1     # the end point is already optimal


def test_homotopy_admm_equals_primal_hot_start():
    """ADMM with the homotopy hot start gives the primal hot start's iterates
    (the per-agent QP solution is unique; here bit for bit, since both end with
    the same final equality-constrained solve)."""
    b = make_workload("ring14")
    r0 = oracle.admm(b, 0, tol=0.0, max_iter=60, start_mode=oracle.START_TURBO)
    r1 = oracle.admm(b, 0, tol=0.0, max_iter=60, start_mode=oracle.START_HOMOTOPY)
    assert r1["homotopy_steps"] > 0
    assert np.array_equal(r0["W"], r1["W"])
    assert np.abs(r0["X"] - r1["X"]).max() <= 1e-12 * max(1.0, np.abs(r0["X"]).max())


def test_heterogeneous_agents_generator_recipe():
    """The mixed-model generator is seeded and gives each agent the damped,
    mass-scaled double integrator it states: p' = p + dt v + dt^2/(2m) u,
    v' = (1 - c dt) v + dt/m u, with c in [0, 0.5) and m in [0.8, 1.25)."""
    from instances import heterogeneous_agents
    b = make_workload("mixed", n_scen=5)
    h1 = heterogeneous_agents(b, seed=4)
    h2 = heterogeneous_agents(b, seed=4)
    assert np.array_equal(h1.A_agent, h2.A_agent) and np.array_equal(h1.B_agent, h2.B_agent)
    na, dp, dt = int(b.N.sum()), b.dp, float(b.A[0, b.dp])
    assert h1.A_agent.shape == (na, b.nx, b.nx) and h1.B_agent.shape == (na, b.nx, b.nu)
    I = np.eye(dp)
    for i in range(na):
        A, B = h1.A_agent[i], h1.B_agent[i]
        c = (1.0 - A[dp, dp]) / dt
        m = dt / B[dp, 0]
        assert 0.0 <= c < 0.5 and 0.8 <= m < 1.25
        assert np.allclose(A[:dp, :dp], I) and np.allclose(A[:dp, dp:], dt * I) and np.allclose(A[dp:, :dp], 0)
        assert np.allclose(A[dp:, dp:], (1 - c * dt) * I)
        assert np.allclose(B[:dp], 0.5 * dt * dt / m * I) and np.allclose(B[dp:], dt / m * I)
    # a subset keeps its agents' models
    sub = h1.subset([1, 3])
    ao = b.agent_off
    assert np.array_equal(sub.A_agent, np.concatenate([h1.A_agent[ao[1]:ao[2]], h1.A_agent[ao[3]:ao[4]]]))


# ----------------------------------------------------------------------------
# Polished point and gradient at an active set with linearly dependent rows
# ----------------------------------------------------------------------------
def _dependent_rows_instance(consistent: bool, seed: int = 3):
    """Five agents, T = 2: all ten pairs are held active at t = 1.  The relative
    positions of five agents span eight dimensions, so at most eight of the ten
    halfspace rows are independent.  The normals at t = 1 are unit vectors with
    a_ij'(pbar_i - pbar_j) = d_min for a reachable configuration pbar, so the
    rows are consistent; with consistent=False one normal is rotated so that
    they are not."""
    rng = np.random.default_rng(seed)
    N, T, dp, dt, d = 5, 2, 2, 0.1, 0.4
    starts = np.array([[0.0, 0.0], [1.2, 0.1], [0.3, 1.1], [-1.0, 0.4], [0.2, -1.3]])
    goals = -starts + 0.1 * rng.standard_normal(starts.shape)
    x_init, x_ref, a, w0, _ = build_scenario(starts, goals, T, dt, d)
    pbar = starts + 0.5 * dt * dt * rng.uniform(-0.8, 0.8, size=starts.shape)
    pl = pair_list(N)
    a = a.reshape(len(pl), T, dp).copy()
    for k, (i, j) in enumerate(pl):
        delta = pbar[i] - pbar[j]
        nd = np.linalg.norm(delta)
        phi = np.arccos(d / nd) * (1 if k % 2 == 0 else -1)
        c, s = np.cos(phi), np.sin(phi)
        a[k, 0] = np.array([[c, -s], [s, c]]) @ (delta / nd)
    if not consistent:
        c, s = np.cos(0.3), np.sin(0.3)
        a[4, 0] = np.array([[c, -s], [s, c]]) @ a[4, 0]
    b = make_batch([dict(N=N, T=T, x_init=x_init, x_ref=x_ref, a=a.reshape(-1, dp), w0=w0, d=d, rho=1.0,
                         umax=1.0, c=None)], dp=dp, dt=dt, umax=1.0)
    act = np.zeros((len(pl), T), dtype=np.uint8)
    act[:, 0] = 1
    W = np.zeros((N, T, 2), dtype=np.int8)
    targets = rng.uniform(-2, 2, size=(N * T, dp))
    return b, act, W, targets


def _numpy_constrained_point(b, act, project: bool):
    """Independent restatement: the global objective of Eq. (1) condensed per
    agent with numpy (tests/helpers), the active halfspace rows G U = d, and the
    minimizer over the affine set by the null-space method (SVD).  With
    project=True d is first replaced by its Euclidean projection onto range(G)."""
    N, T, nx, nu, dp = int(b.N[0]), int(b.T[0]), b.nx, b.nu, b.dp
    pl = pair_list(N)
    Hs, gs, Fs, Gs = [], [], [], []
    for i in range(N):
        Hx = np.array([2 * (b.Qd[i] if t < T else b.Qfd[i]) for t in range(1, T + 1)])
        gx = np.array([-2 * (b.Qd[i] if t < T else b.Qfd[i]) * b.x_ref[i] for t in range(1, T + 1)])
        H, g, F, G = agent_condensed_qp(b.A, b.B, Hx, gx, 2 * b.Rd[i], b.x_init[i])
        Hs.append(H); gs.append(g); Fs.append(F); Gs.append(G)
    n = N * T * nu
    H = np.zeros((n, n)); g = np.zeros(n)
    for i in range(N):
        sl = slice(i * T * nu, (i + 1) * T * nu)
        H[sl, sl] = Hs[i]; g[sl] = gs[i]
    a = b.a.reshape(len(pl), T, dp)
    rows, rhs = [], []
    for k, t in zip(*np.nonzero(act)):
        i, j = pl[k]
        r = np.zeros(n)
        r[i * T * nu:(i + 1) * T * nu] += a[k, t] @ Gs[i][t + 1][:dp]
        r[j * T * nu:(j + 1) * T * nu] -= a[k, t] @ Gs[j][t + 1][:dp]
        rows.append(r)
        rhs.append(b.d_min[0] - a[k, t] @ (Fs[i][t + 1][:dp] - Fs[j][t + 1][:dp]))
    G = np.array(rows); d = np.array(rhs)
    Uu, sv, Vt = np.linalg.svd(G)
    rank = int((sv > 1e-10 * sv[0]).sum())
    if project:
        d = Uu[:, :rank] @ (Uu[:, :rank].T @ d)
    zp = np.linalg.lstsq(G, d, rcond=None)[0]
    Z = Vt[rank:].T
    zu = zp + Z @ np.linalg.solve(Z.T @ H @ Z, -Z.T @ (g + H @ zp))
    X = np.zeros((N, T + 1, nx))
    for i in range(N):
        ui = zu[i * T * nu:(i + 1) * T * nu]
        for t in range(T + 1):
            X[i, t] = Fs[i][t] + Gs[i][t] @ ui
    return X, G, d, rank


@pytest.mark.parametrize("consistent", [True, False])
def test_polished_point_with_dependent_active_rows(consistent):
    b, act, W, targets = _dependent_rows_instance(consistent)
    gr = oracle.global_gradient(b, 0, act, W, targets)
    X, G, d, rank = _numpy_constrained_point(b, act, project=True)
    assert rank == 8 and gr["n_dependent"] == 2
    assert np.abs(gr["X"] - X).max() <= 1e-9 * max(1.0, np.abs(X).max())
    pl = pair_list(5)
    a = b.a.reshape(len(pl), 2, 2)
    viol = np.array([a[k, 0] @ (gr["X"][i, 1, :2] - gr["X"][j, 1, :2]) - b.d_min[0] for k, (i, j) in enumerate(pl)])
    if consistent:
        assert np.abs(viol).max() <= 1e-10          # every active row holds, dependent ones included
    else:
        assert np.abs(viol).max() > 1e-3             # no point satisfies all ten rows
        # the residual of the rows is the least-squares one: orthogonal to their range
        assert np.abs(G.T @ viol).max() <= 1e-10 * max(1.0, np.abs(G).max())


@pytest.mark.parametrize("consistent", [True, False])
def test_gradient_with_dependent_active_rows_matches_central_differences(consistent):
    """Central differences (h = 1e-6) of the loss at the polished point, at the
    same (dependent) active set, against the implicit gradient: diag Q (tied
    Qf), diag R and the goal state of every agent."""
    b, act, W, targets = _dependent_rows_instance(consistent)
    gr = oracle.global_gradient(b, 0, act, W, targets)
    h = 1e-6

    def loss(mod):
        bb = b.subset([0])
        mod(bb)
        return oracle.global_gradient(bb, 0, act, W, targets)["loss"]

    checked = 0
    for i in range(5):
        for r in range(4):
            def mq(bb, s):
                bb.Qd = bb.Qd.copy(); bb.Qfd = bb.Qfd.copy()
                bb.Qd[i, r] += s; bb.Qfd[i, r] += 10 * s

            def mg(bb, s):
                bb.x_ref = bb.x_ref.copy(); bb.x_ref[i, r] += s
            for mod, an in ((mq, gr["gQ"][i, r]), (mg, gr["gGoal"][i, r])):
                fd = (loss(lambda bb: mod(bb, h)) - loss(lambda bb: mod(bb, -h))) / (2 * h)
                assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (i, r, fd, an)
                checked += 1
        for c in range(2):
            def mr(bb, s):
                bb.Rd = bb.Rd.copy(); bb.Rd[i, c] += s
            fd = (loss(lambda bb: mr(bb, h)) - loss(lambda bb: mr(bb, -h))) / (2 * h)
            assert abs(fd - gr["gR"][i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, c, fd, gr["gR"][i, c])
            checked += 1
    assert checked == 50


# ------------------------------------------------------------------ sequential QP over the linearization
def _pair_with_active_collision():
    """The 2-agent crossing with d_min = 1.5 (the generated guess passes the
    agents within 0.97 of each other, so the collision constraint binds)."""
    p = make_workload("pair")
    return dataclasses.replace(p, d_min=np.array([1.5]))


def test_objective_matches_the_global_qp_objective():
    """oracle.objective (numpy) against the C global QP's own objective, which
    leaves out the constant t = 0 state term."""
    for name, n in (("pair", None), ("mixed", 3)):
        b = make_workload(name) if n is None else make_workload(name, n_scen=n)
        for k in range(b.n_scen):
            g = oracle.global_qp(b, k)
            ao = b.agent_off
            e0 = b.x_init[ao[k]:ao[k + 1]] - b.x_ref[ao[k]:ao[k + 1]]
            x0_term = float((e0 * e0 * b.Qd[ao[k]:ao[k + 1]]).sum())
            J = oracle.objective(b, k, g["X"], g["U"])
            assert abs((J - x0_term) - g["obj"]) <= 1e-11 * abs(g["obj"]), (name, k)


def test_min_distance_matches_pairwise_distances():
    from scipy.spatial.distance import pdist
    b = make_workload("mixed", n_scen=3)
    for k in range(b.n_scen):
        o = oracle.admm(b, k, tol=0.0, max_iter=3)
        pos = o["X"][:, 1:, :b.dp]
        want = min(pdist(pos[:, t, :]).min() for t in range(pos.shape[1]))
        assert oracle.min_distance(b, k, o["X"]) == pytest.approx(want, rel=1e-15)


def test_sqp_fixed_point_is_a_local_optimum_of_the_nonconvex_problem():
    """The loop's result on a crossing whose collision constraint binds is a
    local minimizer of Eq. (1) with the exact constraint |p_it - p_jt| >= d_min
    (not its linearization): SLSQP on that nonconvex problem, started at the
    loop's inputs and at a perturbation of them, ends at the same inputs and
    objective.  The stopping rule is also checked on the recorded objectives."""
    p = _pair_with_active_collision()
    r = oracle.sqp(p, 0, tol=1e-9, max_iter=20000, max_outer=30, obj_rtol=1e-12)
    assert r["sqp_status"] == 0 and r["status"] == oracle.CONVERGED and r["outer"] >= 3
    Js = r["objectives"]
    assert abs(Js[-1] - Js[-2]) <= 1e-12 * abs(Js[-2])
    assert all(abs(Js[m] - Js[m - 1]) > 1e-12 * abs(Js[m - 1]) for m in range(1, len(Js) - 1))
    assert r["min_dist"] == pytest.approx(1.5, abs=1e-7)

    N, T, nx, nu = 2, int(p.T[0]), p.nx, p.nu
    A, B = p.A.reshape(nx, nx), p.B.reshape(nx, nu)

    def states(u):
        u = u.reshape(N, T, nu)
        X = np.zeros((N, T + 1, nx))
        X[:, 0] = p.x_init
        for t in range(T):
            X[:, t + 1] = X[:, t] @ A.T + u[:, t] @ B.T
        return X

    def cost(u):
        X, uu = states(u), u.reshape(N, T, nu)
        e = X - p.x_ref[:, None, :]
        return (e[:, :T] ** 2 * p.Qd[:, None, :]).sum() + (uu ** 2 * p.Rd[:, None, :]).sum() + \
            (e[:, T] ** 2 * p.Qfd).sum()

    def separation(u):
        d = states(u)[0, 1:, :2] - states(u)[1, 1:, :2]
        return (d * d).sum(axis=1) - 1.5 ** 2

    bounds = [(p.umin[c % nu], p.umax[c % nu]) for c in range(N * T * nu)]
    u_sqp = r["U"].ravel()
    assert cost(u_sqp) == pytest.approx(r["objective"], rel=1e-13)
    rng = np.random.default_rng(5)
    for u0 in (u_sqp, np.clip(u_sqp + 0.05 * rng.standard_normal(u_sqp.size), -1.0, 1.0)):
        res = minimize(cost, u0, method="SLSQP", bounds=bounds, constraints=[{"type": "ineq", "fun": separation}],
                       options=dict(ftol=1e-14, maxiter=1000))
        assert res.fun >= r["objective"] * (1 - 1e-9)
        assert abs(res.fun - r["objective"]) <= 1e-9 * r["objective"]
        assert np.abs(res.x - u_sqp).max() <= 1e-4


def test_sqp_stops_at_once_when_the_collision_constraint_is_slack():
    """The stock crossing never comes within d_min = 0.5: the relinearized QP
    has the same solution, so the loop stops at the second step with an
    objective change at rounding level."""
    p = make_workload("pair")
    r = oracle.sqp(p, 0, tol=1e-4, max_iter=500, max_outer=5)
    assert r["outer"] == 2 and r["sqp_status"] == 0
    assert r["min_dist"] > 0.5
    assert r["objectives"][1] == pytest.approx(r["objectives"][0], rel=1e-9)
