"""Implicit-KKT adjoint (tadmm_backward) against the oracle's dense-KKT gradient
and central finite differences.

Both sides take the active set from their own run (bound working sets of the
last x-update, halfspaces with theta > 1e-9); the per-iteration parity makes
them equal, which the tests assert before comparing.  FP64 gradients within
1e-6 relative of the oracle, FP32 within 1e-3 relative (against the FP64
oracle); the polished states within 1e-9 (FP64).
"""
import numpy as np
import pytest

import oracle
from instances import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_15838_gb300 import build
    build.build()
    import paper_2602_15838_gb300 as m
    return m


def _loss_grad(b, X, targets):
    """loss = sum ||p_it - target_it||^2 over t = 1..T and its gradient wrt packed X."""
    g = np.zeros_like(X)
    loss = 0.0
    xo = 0
    to = 0
    for k in range(b.n_scen):
        N, T = int(b.N[k]), int(b.T[k])
        Xk = X[xo:xo + N * (T + 1) * b.nx].reshape(N, T + 1, b.nx)
        tk = targets[to:to + N * T].reshape(N, T, b.dp)
        e = Xk[:, 1:, :b.dp] - tk
        loss += float((e ** 2).sum())
        gk = np.zeros_like(Xk)
        gk[:, 1:, :b.dp] = 2 * e
        g[xo:xo + gk.size] = gk.ravel()
        xo += gk.size
        to += N * T
    return loss, g


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1.0, np.abs(np.asarray(b)).max()))


def _case(N, T, n_scen=2, knn=None, hetero=False):
    b = make_workload("diff", n_scen=n_scen, N_override=N, T_override=T)
    if knn is not None:
        from instances import nearest_neighbour_pairs
        b = nearest_neighbour_pairs(b, knn)
    if hetero:
        from instances import heterogeneous_agents
        b = heterogeneous_agents(b, seed=11)
    return b


@pytest.mark.parametrize("precision,tol,N,T,iters,n_scen,knn,hetero", [
    (64, 1e-6, 6, 12, 40, 2, None, False), (64, 1e-6, 10, 20, 300, 2, None, False),
    (32, 1e-3, 6, 12, 40, 2, None, False), (32, 1e-3, 10, 20, 300, 2, None, False),
    (64, 1e-6, 10, 20, 300, 2, 3, False), (64, 1e-6, 10, 20, 300, 2, None, True)])
def test_gradient_matches_oracle_dense_kkt(tg, precision, tol, N, T, iters, n_scen, knn, hetero):
    """(knn: coupling only each agent's knn nearest neighbours; hetero: per-agent
    dynamics.)"""
    b = _case(N, T, n_scen, knn, hetero)
    s = tg.Solver(b, precision=precision)
    s.solve(0.0, iters)
    sol = s.solution()
    out = s.split(sol)
    _, gX = _loss_grad(b, np.asarray(sol["X"]), b.targets)
    # the loss gradient is taken at the polished solution on both sides
    pol = s.backward(np.zeros_like(gX))
    loss, gX = _loss_grad(b, pol["X_polished"], b.targets)
    g = s.backward(gX)
    assert (g["status"] == 0).all()
    ao = b.agent_off
    xo = 0
    for k in range(b.n_scen):
        N, T = int(b.N[k]), int(b.T[k])
        o = oracle.admm(b, k, tol=0.0, max_iter=iters, nthreads=8)
        act_o = o["theta"] > 1e-9
        act_g = out[k]["theta"] > 1e-9
        if precision == 64:
            assert np.array_equal(act_o, act_g)
            assert np.array_equal(o["W"], out[k]["W"])
        elif not (np.array_equal(act_o, act_g) and np.array_equal(o["W"], out[k]["W"])):
            xo += N * (T + 1) * b.nx
            continue   # float32 iterates may flip a threshold decision; nothing to compare
        tk = b.targets[int(b.agentstep_off[k]):int(b.agentstep_off[k + 1])]
        ref = oracle.global_gradient(b, k, act_o.astype(np.uint8), o["W"], tk, qf_tie=10.0)
        Xp = pol["X_polished"][xo:xo + N * (T + 1) * b.nx].reshape(N, T + 1, b.nx)
        assert _rel(Xp, ref["X"]) <= (1e-9 if precision == 64 else 1e-4)
        sl = slice(int(ao[k]), int(ao[k + 1]))
        gq = g["gQ"][sl] + 10.0 * g["gQf"][sl]
        assert _rel(gq, ref["gQ"]) <= tol
        assert _rel(g["gR"][sl], ref["gR"]) <= tol
        assert _rel(g["gGoal"][sl], ref["gGoal"]) <= tol
        xo += N * (T + 1) * b.nx
    s.close()


def test_gradient_full_size_differentiation_scenario_fp64(tg):
    """A 16-agent, T = 30 scenario of the differentiation workload after 1000
    iterations (about 100 active halfspaces, not yet the optimal active set at
    rho = 1): the Schur complement is ill-conditioned, so the polished solution
    is checked through its own equality residual and both gradients agree to
    the conditioning-limited 1e-4."""
    b = make_workload("diff", n_scen=1)
    iters = 1000
    s = tg.Solver(b, precision=64)
    s.solve(0.0, iters)
    out = s.split(s.solution())[0]
    pol = s.backward(np.zeros(s.sizes["X"]))
    loss, gX = _loss_grad(b, pol["X_polished"], b.targets)
    g = s.backward(gX)
    assert (g["status"] == 0).all()
    N, T = int(b.N[0]), int(b.T[0])
    P = N * (N - 1) // 2
    Xp = pol["X_polished"].reshape(N, T + 1, b.nx)
    act = out["theta"] > 1e-9
    from instances import pair_list
    pl = pair_list(N)
    a = b.a.reshape(P, T, 2)
    res = []
    for k, t in zip(*np.nonzero(act)):
        i, j = pl[k]
        res.append(abs(a[k, t] @ (Xp[i, t + 1, :2] - Xp[j, t + 1, :2]) - b.d_min[0]))
    assert len(res) > 20 and max(res) <= 1e-8 * max(1.0, np.abs(Xp).max())
    o = oracle.admm(b, 0, tol=0.0, max_iter=iters, nthreads=8)
    assert np.array_equal(o["theta"] > 1e-9, act) and np.array_equal(o["W"], out["W"])
    ref = oracle.global_gradient(b, 0, act.astype(np.uint8), o["W"], b.targets, qf_tie=10.0)
    assert _rel(Xp, ref["X"]) <= 1e-4
    assert _rel(g["gQ"] + 10 * g["gQf"], ref["gQ"]) <= 1e-4
    assert _rel(g["gR"], ref["gR"]) <= 1e-4
    assert _rel(g["gGoal"], ref["gGoal"]) <= 1e-4
    s.close()


def test_gradient_matches_central_differences_fp64(tg):
    """Central differences (h = 1e-6) of the loss at the polished solution,
    re-solving with perturbed parameters; entries whose active set changes at
    +-h are skipped."""
    b = _case(5, 10, n_scen=1)
    iters = 40
    s = tg.Solver(b, precision=64)

    def run(bb):
        s.update(bb)
        s.solve(0.0, iters)
        sol = s.split(s.solution())[0]
        pol = s.backward(np.zeros(s.sizes["X"]))
        loss, gX = _loss_grad(bb, pol["X_polished"], bb.targets)
        return loss, gX, sol["theta"] > 1e-9, sol["W"]

    loss0, gX, act0, W0 = run(b)
    g = s.backward(gX)
    h = 1e-6
    checked = 0
    for i in range(5):
        for r in range(4):
            for kind in ("Q", "goal"):
                vals = []
                for sgn in (1, -1):
                    bb = b.subset([0])
                    if kind == "Q":
                        bb.Qd = bb.Qd.copy(); bb.Qfd = bb.Qfd.copy()
                        bb.Qd[i, r] += sgn * h; bb.Qfd[i, r] += sgn * 10 * h
                    else:
                        bb.x_ref = bb.x_ref.copy(); bb.x_ref[i, r] += sgn * h
                    l, _, act, W = run(bb)
                    vals.append((l, np.array_equal(act, act0) and np.array_equal(W, W0)))
                if not (vals[0][1] and vals[1][1]):
                    continue
                fd = (vals[0][0] - vals[1][0]) / (2 * h)
                an = g["gQ"][i, r] + 10 * g["gQf"][i, r] if kind == "Q" else g["gGoal"][i, r]
                assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (kind, i, r, fd, an)
                checked += 1
    assert checked >= 20
    s.close()


def test_autograd_function(tg):
    import torch
    b = _case(4, 10, n_scen=1)
    s = tg.Solver(b, precision=64)
    Qd = torch.tensor(b.Qd, dtype=torch.float64, requires_grad=True)
    Rd = torch.tensor(b.Rd, dtype=torch.float64, requires_grad=True)
    goal = torch.tensor(b.x_ref, dtype=torch.float64, requires_grad=True)
    X = tg.TADMMFunction.apply(Qd, Rd, goal, s, 0.0, 40)
    N, T = int(b.N[0]), int(b.T[0])
    tgt = torch.tensor(b.targets.reshape(N, T, 2))
    loss = ((X.view(N, T + 1, b.nx)[:, 1:, :2].cpu() - tgt) ** 2).sum()
    loss.backward()
    assert Qd.grad is not None and torch.isfinite(Qd.grad).all()
    assert Rd.grad.abs().sum() > 0 and goal.grad.abs().sum() > 0
    s.close()
