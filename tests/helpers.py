"""Independent numpy formulations used to pin the oracle (no oracle code here)."""
import numpy as np


def condensed(A, B, x0, T):
    """Free response F[t] (t = 0..T) and input-to-state maps G[t] (t = 0..T, [nx, T*nu])
    built by simulating unit impulses."""
    nx, nu = B.shape
    F = np.zeros((T + 1, nx))
    F[0] = x0
    for t in range(T):
        F[t + 1] = A @ F[t]
    G = np.zeros((T + 1, nx, T * nu))
    for k in range(T * nu):
        u = np.zeros(T * nu)
        u[k] = 1.0
        x = np.zeros(nx)
        for t in range(T):
            x = A @ x + B @ u[t * nu:(t + 1) * nu]
            G[t + 1, :, k] = x
    return F, G


def agent_condensed_qp(A, B, Hx, gx, Hu, x0):
    """Hessian and gradient of the per-agent QP as a function of the stacked inputs."""
    T = Hx.shape[0]
    F, G = condensed(A, B, x0, T)
    nu = B.shape[1]
    H = np.kron(np.eye(T), np.diag(Hu)).astype(float)
    g = np.zeros(T * nu)
    for t in range(1, T + 1):
        Gt = G[t]
        H += Gt.T @ np.diag(Hx[t - 1]) @ Gt
        g += Gt.T @ (np.diag(Hx[t - 1]) @ F[t] + gx[t - 1])
    return H, g, F, G


def random_agent_qp(rng, T, nx=4, nu=2, box=1.0, double_integrator=True):
    if double_integrator:
        dp = nx // 2
        dt = 0.1
        A = np.block([[np.eye(dp), dt * np.eye(dp)], [np.zeros((dp, dp)), np.eye(dp)]])
        B = np.vstack([0.5 * dt * dt * np.eye(dp), dt * np.eye(dp)])
    else:
        A = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx))
        B = rng.standard_normal((nx, nu))
    Hx = 0.2 + 3.0 * rng.random((T, nx))
    gx = 20.0 * rng.standard_normal((T, nx))
    Hu = 0.2 + rng.random(nu)
    x0 = rng.standard_normal(nx)
    umin = -box * (0.5 + rng.random(nu))
    umax = box * (0.5 + rng.random(nu))
    return A, B, Hx, gx, Hu, x0, umin, umax


def costate_gradient(A, B, Hx, gx, Hu, x, u):
    """Gradient of the per-agent objective with respect to u_t through the adjoint
    recursion lam_T = Hx_T x_T + gx_T, lam_t = Hx_t x_t + gx_t + A' lam_{t+1}."""
    T = Hx.shape[0]
    lam = np.zeros((T + 2, A.shape[0]))
    for t in range(T, 0, -1):
        lam[t] = Hx[t - 1] * x[t] + gx[t - 1] + (A.T @ lam[t + 1] if t < T else 0.0)
    grad = np.zeros_like(u)
    for t in range(T):
        grad[t] = Hu * u[t] + B.T @ lam[t + 1]
    return grad
