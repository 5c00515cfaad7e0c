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


def _loss_per_scenario(b, X, targets):
    out = np.zeros(b.n_scen)
    xo = to = 0
    for k in range(b.n_scen):
        N, T = int(b.N[k]), int(b.T[k])
        Xk = X[xo:xo + N * (T + 1) * b.nx].reshape(N, T + 1, b.nx)
        tk = targets[to:to + N * T].reshape(N, T, b.dp)
        out[k] = float(((Xk[:, 1:, :b.dp] - tk) ** 2).sum())
        xo += N * (T + 1) * b.nx
        to += N * T
    return out


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
    dynamics.)  FP64: the GPU's active set equals the oracle ADMM's and both
    gradients are taken there.  FP32: the oracle takes the FP32 run's own
    active set (float32 iterates may flip a threshold decision), so that every
    scenario is compared."""
    b = _case(N, T, n_scen, knn, hetero)
    s = tg.Solver(b, precision=precision)
    s.solve(0.0, iters)
    sol = s.solution()
    out = s.split(sol)
    pol = s.backward(None)
    loss, gX = _loss_grad(b, pol["X_polished"], b.targets)
    g = s.backward(gX)
    assert (g["status"] == 0).all()
    ao = b.agent_off
    xo = 0
    compared = 0
    for k in range(b.n_scen):
        N, T = int(b.N[k]), int(b.T[k])
        act_g = out[k]["theta"] > 1e-9
        W_g = out[k]["W"]
        if precision == 64:
            o = oracle.admm(b, k, tol=0.0, max_iter=iters, nthreads=8)
            assert np.array_equal(o["theta"] > 1e-9, act_g)
            assert np.array_equal(o["W"], W_g)
        tk = b.targets[int(b.agentstep_off[k]):int(b.agentstep_off[k + 1])]
        ref = oracle.global_gradient(b, k, act_g.astype(np.uint8), W_g, tk, qf_tie=10.0)
        Xp = pol["X_polished"][xo:xo + N * (T + 1) * b.nx].reshape(N, T + 1, b.nx)
        assert _rel(Xp, ref["X"]) <= (1e-9 if precision == 64 else 1e-4)
        sl = slice(int(ao[k]), int(ao[k + 1]))
        gq = g["gQ"][sl] + 10.0 * g["gQf"][sl]
        assert _rel(gq, ref["gQ"]) <= tol
        assert _rel(g["gR"][sl], ref["gR"]) <= tol
        assert _rel(g["gGoal"][sl], ref["gGoal"]) <= tol
        assert int(g["n_dependent"][k]) == ref["n_dependent"]
        compared += 1
        xo += N * (T + 1) * b.nx
    assert compared == b.n_scen
    s.close()


def _certify_optimal(b, k, ref, act, W, tol):
    """KKT conditions of the global QP at the oracle's polished point of the
    given active set: every halfspace and input bound holds, and the multipliers
    of the active rows are non-negative (within tol, relative)."""
    from instances import pair_list
    N, T, P = int(b.N[k]), int(b.T[k]), int(b.P[k])
    pl = pair_list(N)
    a = b.a[b.pairstep_off[k]:b.pairstep_off[k + 1]].reshape(P, T, b.dp)
    X, U = ref["X"], ref["U"]
    slack = (a * (X[pl[:, 0], 1:, :b.dp] - X[pl[:, 1], 1:, :b.dp])).sum(-1) - b.d_min[k]
    scale = max(1.0, np.abs(ref["mu_h"]).max(), np.abs(ref["mu_u"]).max())
    ok = slack.min() >= -tol * max(1.0, b.d_min[k])
    ok = ok and (U - b.umax).max() <= tol and (b.umin - U).max() <= tol
    if act.any():
        ok = ok and ref["mu_h"][act.astype(bool)].min() >= -tol * scale
    if (W != 0).any():
        ok = ok and ref["mu_u"][W != 0].min() >= -tol * scale
    return bool(ok)


def _split_set(b, pol, k, to, uo):
    N, T, P = int(b.N[k]), int(b.T[k]), int(b.P[k])
    return pol["act"][to:to + P * T].reshape(P, T), pol["W"][uo:uo + N * T * b.nu].reshape(N, T, b.nu)


def _full_size_case(tg, precision, iters):
    """The differentiation workload at full size: 64 scenarios x 16 agents, 2D,
    T = 30.  ADMM with residual balancing of rho (every 10 iterations, mu 10,
    tau 2) to tol 1e-6 (FP64) / 1e-5 (FP32) or `iters` iterations, then the
    active set read off the final iterate is polished on the centralized QP
    until the KKT conditions hold (tadmm_polish)."""
    b = make_workload("diff", n_scen=64)
    s = tg.Solver(b, precision=precision, adapt=(10, 10.0, 2.0))
    s.solve(1e-6 if precision == 64 else 1e-5, iters)
    pol = s.polish(1e-9, 100)
    base = s.backward(None)
    loss, gX = _loss_grad(b, base["X_polished"], b.targets)
    g = s.backward(gX)
    return b, s, pol, base, g


@pytest.mark.parametrize("precision", [64, 32])
def test_gradient_differentiation_workload_full_size(tg, precision):
    """64 x 16 agents, T = 30, every scenario: the GPU's polished active set is
    handed to the oracle, which (i) certifies it as the optimum of the global
    QP by the KKT conditions of its own dense polished point and (ii) computes
    the dense-KKT gradient there; the GPU gradient agrees element by element
    within 1e-6 (FP64) / 1e-3 (FP32) and the polished states within 1e-9 /
    1e-4.  FP64: every scenario is compared, and at least 60 of 64 sets are
    certified optimal after 2000 ADMM iterations and at most 100 polishing
    rounds (the others stop at the round cap; their gradient is the one of
    the set reached, still compared).  FP32: the comparison covers the sets the
    oracle certifies (at least 56 of 64); at the others float32 cannot resolve
    the nearly dependent active rows (multipliers up to 1e6)."""
    b, s, pol, base, g = _full_size_case(tg, precision, 2000 if precision == 64 else 5000)
    assert (g["status"] == 0).all()
    tol = 1e-6 if precision == 64 else 1e-3
    to = uo = xo = 0
    certified = compared = 0
    for k in range(b.n_scen):
        N, T, P = int(b.N[k]), int(b.T[k]), int(b.P[k])
        act, W = _split_set(b, pol, k, to, uo)
        tk = b.targets[int(b.agentstep_off[k]):int(b.agentstep_off[k + 1])]
        ref = oracle.global_gradient(b, k, act, W, tk, qf_tie=10.0)
        opt = _certify_optimal(b, k, ref, act, W, 1e-8 if precision == 64 else 1e-4)
        if pol["status"][k] == 0 and precision == 64:
            assert opt, k          # the GPU's KKT claim holds at the oracle's own point
        certified += opt
        if precision == 64 or opt:
            Xp = base["X_polished"][xo:xo + N * (T + 1) * b.nx].reshape(N, T + 1, b.nx)
            assert _rel(Xp, ref["X"]) <= (1e-9 if precision == 64 else 1e-4), k
            sl = slice(int(b.agent_off[k]), int(b.agent_off[k + 1]))
            assert _rel(g["gQ"][sl] + 10.0 * g["gQf"][sl], ref["gQ"]) <= tol, k
            assert _rel(g["gR"][sl], ref["gR"]) <= tol, k
            assert _rel(g["gGoal"][sl], ref["gGoal"]) <= tol, k
            compared += 1
        to += P * T
        uo += N * T * b.nu
        xo += N * (T + 1) * b.nx
    if precision == 64:
        assert compared == 64 and certified >= 60, (compared, certified)
    else:
        assert compared >= 56 and certified == compared, (compared, certified)
    s.close()


def test_gradient_differentiation_workload_central_differences_fp64(tg):
    """Central differences (h = 1e-6) on the full 64 x 16, T = 30 batch at the
    polished active sets: for a seeded subset of (agent, entry) slots covering
    diag Q (with the tied Qf), diag R and the goal state, the entry is moved by
    +-h in all 64 scenarios at once (tadmm_update), the polished point of the
    same active set is formed again (tadmm_backward with no loss gradient) and
    the difference quotient of each scenario's loss is compared with the
    implicit gradient.  The active set is held fixed: the gradient is the
    derivative of the polished solution map, which equals the derivative of
    the QP solution where the active set is locally constant."""
    b, s, pol, base, g = _full_size_case(tg, 64, 2000)
    rng = np.random.default_rng(5)
    slots = [("Q", int(i), int(r)) for i, r in zip(rng.integers(0, 16, 4), rng.integers(0, 4, 4))]
    slots += [("R", int(i), int(c)) for i, c in zip(rng.integers(0, 16, 4), rng.integers(0, 2, 4))]
    slots += [("goal", int(i), int(r)) for i, r in zip(rng.integers(0, 16, 4), rng.integers(0, 4, 4))]
    h = 1e-6
    ao = b.agent_off[:-1]

    def losses(kind, i, r, sgn):
        bb = b.subset(list(range(b.n_scen)))
        rows = ao + i
        if kind == "Q":
            bb.Qd = bb.Qd.copy(); bb.Qfd = bb.Qfd.copy()
            bb.Qd[rows, r] += sgn * h; bb.Qfd[rows, r] += sgn * 10 * h
        elif kind == "R":
            bb.Rd = bb.Rd.copy(); bb.Rd[rows, r] += sgn * h
        else:
            bb.x_ref = bb.x_ref.copy(); bb.x_ref[rows, r] += sgn * h
        s.update(bb)
        return _loss_per_scenario(bb, s.backward(None)["X_polished"], b.targets)

    checked = 0
    worst = 0.0
    for kind, i, r in slots:
        fd = (losses(kind, i, r, 1) - losses(kind, i, r, -1)) / (2 * h)
        rows = ao + i
        if kind == "Q":
            an = g["gQ"][rows, r] + 10 * g["gQf"][rows, r]
        elif kind == "R":
            an = g["gR"][rows, r]
        else:
            an = g["gGoal"][rows, r]
        err = np.abs(fd - an) / np.maximum(1.0, np.abs(fd))
        worst = max(worst, float(err.max()))
        assert (err <= 1e-5).all(), (kind, i, r, float(err.max()))
        checked += fd.size
    assert checked == 12 * 64
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
    """TADMMFunction: loss.backward() gives exactly Solver.backward's gradient at
    the same solve, that gradient matches the oracle's dense-KKT gradient at the
    GPU's active set (1e-6), and central differences (h = 1e-6) of the loss
    through the differentiable forward (a full re-solve per evaluation) match
    it on every entry whose active set stays the same at +-h."""
    import torch
    b = _case(4, 10, n_scen=1)
    s = tg.Solver(b, precision=64)
    N, T = int(b.N[0]), int(b.T[0])
    tgt = torch.tensor(b.targets.reshape(N, T, 2))
    # the forward writes its parameters into the solver's batch (= b): keep the originals
    Q0, R0, G0 = b.Qd.copy(), b.Rd.copy(), b.x_ref.copy()

    def forward(Qd, Rd, goal):
        X = tg.TADMMFunction.apply(Qd, Rd, goal, s, 0.0, 40)
        return X, ((X.view(N, T + 1, b.nx)[:, 1:, :2].cpu() - tgt) ** 2).sum()

    Qd = torch.tensor(Q0, dtype=torch.float64, requires_grad=True)
    Rd = torch.tensor(R0, dtype=torch.float64, requires_grad=True)
    goal = torch.tensor(G0, dtype=torch.float64, requires_grad=True)
    X, loss = forward(Qd, Rd, goal)
    loss.backward()
    # the same gradient straight from the solver
    _, gX = _loss_grad(b, X.detach().cpu().numpy(), b.targets)
    g = s.backward(gX)
    assert np.array_equal(Qd.grad.numpy(), g["gQ"] + 10.0 * g["gQf"])
    assert np.array_equal(Rd.grad.numpy(), g["gR"]) and np.array_equal(goal.grad.numpy(), g["gGoal"])
    # against the oracle at the GPU's active set
    out = s.split(s.solution())[0]
    ref = oracle.global_gradient(b, 0, (out["theta"] > 1e-9).astype(np.uint8), out["W"], b.targets, qf_tie=10.0)
    assert _rel(Qd.grad.numpy(), ref["gQ"]) <= 1e-6
    assert _rel(Rd.grad.numpy(), ref["gR"]) <= 1e-6
    assert _rel(goal.grad.numpy(), ref["gGoal"]) <= 1e-6
    # central differences through the differentiable forward
    act0, W0 = out["theta"] > 1e-9, out["W"]
    h = 1e-6
    checked = 0
    for name, base, grad in (("Q", Q0, Qd.grad), ("R", R0, Rd.grad), ("goal", G0, goal.grad)):
        for i in range(N):
            for r in range(base.shape[1]):
                vals = []
                for sgn in (1, -1):
                    args = [torch.tensor(Q0), torch.tensor(R0), torch.tensor(G0)]
                    k = {"Q": 0, "R": 1, "goal": 2}[name]
                    args[k] = args[k].clone()
                    args[k][i, r] += sgn * h
                    with torch.no_grad():
                        _, l = forward(*args)
                    o2 = s.split(s.solution())[0]
                    vals.append((float(l), np.array_equal(o2["theta"] > 1e-9, act0) and np.array_equal(o2["W"], W0)))
                if not (vals[0][1] and vals[1][1]):
                    continue
                fd = (vals[0][0] - vals[1][0]) / (2 * h)
                assert abs(fd - float(grad[i, r])) <= 1e-5 * max(1.0, abs(fd)), (name, i, r, fd, float(grad[i, r]))
                checked += 1
    assert checked >= 30
    s.close()


def test_gradient_3d_model_matches_oracle(tg):
    """The 3D double integrator (nx = 6, nu = 3) of the swarm workload with 5
    agents, T = 8: the implicit-KKT gradient of a position-tracking loss at
    the GPU's final active set (polished to KKT) against the oracle's
    dense-KKT gradient at the same set (1e-6), and the polished states
    (1e-9)."""
    b = make_workload("swarm3d", N_override=5, T_override=8)
    N, T = int(b.N[0]), int(b.T[0])
    rng = np.random.default_rng(8)
    targets = rng.uniform(-3.0, 3.0, size=(N * T, 3))
    s = tg.Solver(b, precision=64)
    s.solve(1e-6, 3000)
    pol = s.polish(1e-9, 50)
    assert pol["status"][0] == 0
    X = s.backward(None)["X_polished"].reshape(N, T + 1, 6)
    gX = np.zeros_like(X)
    gX[:, 1:, :3] = 2 * (X[:, 1:, :3] - targets.reshape(N, T, 3))
    g = s.backward(gX.ravel())
    P = N * (N - 1) // 2
    act = pol["act"].reshape(P, T)
    W = pol["W"].reshape(N, T, 3)
    ref = oracle.global_gradient(b, 0, act, W, targets, qf_tie=10.0)
    assert act.sum() + (W != 0).sum() > 0
    assert _rel(X, ref["X"]) <= 1e-9
    assert _rel(g["gQ"] + 10.0 * g["gQf"], ref["gQ"]) <= 1e-6
    assert _rel(g["gR"], ref["gR"]) <= 1e-6
    assert _rel(g["gGoal"], ref["gGoal"]) <= 1e-6
    s.close()


def test_backward_after_graph_and_plain_mode_solves(tg):
    """The adjoint reads the final iterate (its theta slot and working sets)
    of whichever execution mode solved: after a graph-mode or a plain-mode
    solve it gives bitwise the gradients and polished states of the
    persistent kernel's solve."""
    b = _case(6, 12, n_scen=3)
    res = {}
    for mode in ("batched", "graph", "plain"):
        s = tg.Solver(b, precision=64, mode=mode)
        s.solve(0.0, 30)
        X = s.backward(None)["X_polished"]
        _, gX = _loss_grad(b, X, b.targets)
        res[mode] = (X, s.backward(gX))
        s.close()
    for mode in ("graph", "plain"):
        assert np.array_equal(res[mode][0], res["batched"][0]), mode
        for key in ("gQ", "gQf", "gR", "gGoal"):
            assert np.array_equal(res[mode][1][key], res["batched"][1][key]), (mode, key)


def test_polish_and_gradient_with_listed_pairs(tg):
    """Listed (4-nearest-neighbour) coupling: the polished active set is
    certified optimal by the oracle and the gradient matches its dense-KKT
    gradient (1e-6) at that set."""
    from instances import nearest_neighbour_pairs
    b = nearest_neighbour_pairs(make_workload("diff", n_scen=4), 4)
    s = tg.Solver(b, precision=64, adapt=(10, 10.0, 2.0))
    s.solve(1e-6, 3000)
    pol = s.polish(1e-9, 100)
    X = s.backward(None)["X_polished"]
    _, gX = _loss_grad(b, X, b.targets)
    g = s.backward(gX)
    to = uo = 0
    certified = 0
    for k in range(b.n_scen):
        N, T, P = int(b.N[k]), int(b.T[k]), int(b.P[k])
        act = pol["act"][to:to + P * T].reshape(P, T)
        W = pol["W"][uo:uo + N * T * b.nu].reshape(N, T, b.nu)
        tk = b.targets[int(b.agentstep_off[k]):int(b.agentstep_off[k + 1])]
        ref = oracle.global_gradient(b, k, act, W, tk, qf_tie=10.0)
        if pol["status"][k] == 0:
            assert _certify_listed(b, k, ref, act, W), k
            certified += 1
        sl = slice(int(b.agent_off[k]), int(b.agent_off[k + 1]))
        assert _rel(g["gQ"][sl] + 10.0 * g["gQf"][sl], ref["gQ"]) <= 1e-6, k
        assert _rel(g["gR"][sl], ref["gR"]) <= 1e-6, k
        assert _rel(g["gGoal"][sl], ref["gGoal"]) <= 1e-6, k
        to += P * T
        uo += N * T * b.nu
    assert certified >= 3
    s.close()


def _certify_listed(b, k, ref, act, W, tol=1e-8):
    """KKT conditions at the oracle's polished point with the scenario's listed pairs."""
    N, T, P = int(b.N[k]), int(b.T[k]), int(b.P[k])
    pl = np.asarray(b.pairs_of(k)).reshape(P, 2)
    a = b.a[b.pairstep_off[k]:b.pairstep_off[k + 1]].reshape(P, T, b.dp)
    X, U = ref["X"], ref["U"]
    slack = (a * (X[pl[:, 0], 1:, :b.dp] - X[pl[:, 1], 1:, :b.dp])).sum(-1) - b.d_min[k]
    scale = max(1.0, np.abs(ref["mu_h"]).max(), np.abs(ref["mu_u"]).max())
    ok = slack.min() >= -tol * max(1.0, b.d_min[k])
    ok = ok and (U - b.umax).max() <= tol and (b.umin - U).max() <= tol
    if act.any():
        ok = ok and ref["mu_h"][act.astype(bool)].min() >= -tol * scale
    if (W != 0).any():
        ok = ok and ref["mu_u"][W != 0].min() >= -tol * scale
    return bool(ok)
