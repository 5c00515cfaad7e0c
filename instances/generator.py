"""Seeded generator of multi-agent collision-avoidance QP instances.

Workload shapes follow the paper's benchmark family (2D double integrator
agents crossing a shared workspace with dense all-pairs collision coupling,
Sec. V.A) at five synthetic sizes (make_workload names):

  "pair"        N=2 agents on a radius-5 circle, antipodal goals, jitter
                sigma 0.05, T=20, d_min=0.5, rho=1.
  "ring14"      N=14 agents on a radius-5 circle, antipodal goals, jitter
                sigma 0.1, T=20, d_min=0.5, rho=1.
  "mixed"       a batch of scenarios with N ~ U{2..32}, T ~ U{20..40}; starts
                uniform in [-5,5]^2 (rejection-sampled >= 2*d_min apart), goals
                a random permutation of the starts; d_min=0.4, rho=1.
  "swarm3d"     N=512 3D double integrators, T=40, |u|<=2, starts uniform in
                [-20,20]^3 (>= 2*d_min apart), goals = -starts; d_min=0.5, rho=2.
  "diff"        64 scenarios x 16 agents, T=30, drawn as "mixed", plus seeded
                position targets uniform in [-5,5]^2 for a tracking loss.

Collision linearization (Sec. III.A: the distance constraint is replaced by a
halfspace built from reference trajectories; the references are straight
constant-velocity lines, Sec. V.A).  The straight-line guess of agent i is
its zero-input trajectory from x_init = [s_i; v0_i] with
v0_i = c * (goal_i - s_i) / (T dt), i.e. g_{i,t} = s_i + c (t/T)(goal_i - s_i).
c is the largest value in {1, 1/2, ..., 2^-20, 0} for which every pair keeps
at least 1.1*d_min separation over t = 1..T.  The halfspace normal is the unit
vector a_ijt = (g_it - g_jt)/||g_it - g_jt||, and the constraint is
a_ijt^T (p_it - p_jt) >= d_min.  The guess satisfies every halfspace, so each
instance is feasible by construction.  The `literal` variant (zero initial
velocity, c = 1 lines) is generally infeasible and serves as a negative case.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) as a counter-based
stream, output n = mix(seed + (n+1) * 0x9E3779B97F4A7C15); uniforms are the
top 53 bits; normals by Box-Muller.  Stream seed for scenario k of workload
stream id c (1..5 in the order listed above) is (c << 32) + k, so the first k
scenarios of a batch do not depend on its size.

Packed batch layout (all float64 unless stated; row-major):
  N[S], T[S]                 int32 agent count and horizon per scenario
  A[nx,nx], B[nx,nu]         shared model; umin[nu], umax[nu] shared box
  Qd, Qfd [sum N, nx]; Rd [sum N, nu]   per-agent diagonal weights
  x_init, x_ref [sum N, nx]  initial state and (constant) goal state
  a  [sum_s P_s T_s, dp]     halfspace normals, scenario-major, then pair
                             (lexicographic i<j), then t = 1..T
  w0 [sum_s N_s T_s, dp]     initial consensus positions (the guesses),
                             scenario, agent, t = 1..T
  d_min[S], rho[S]
  targets [sum_s N_s T_s, dp] ("diff" only) loss targets
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream (vectorised over the counter)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.n = 0

    def next_u64(self, k: int) -> np.ndarray:
        idx = np.arange(self.n + 1, self.n + k + 1, dtype=np.uint64)
        self.n += k
        with np.errstate(over="ignore"):
            z = self.seed + idx * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int) -> np.ndarray:
        return (self.next_u64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, k: int) -> np.ndarray:
        u = self.uniform(2 * k).reshape(k, 2)
        return np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in {lo, ..., hi}."""
        return lo + int(self.uniform(1)[0] * (hi - lo + 1))


def double_integrator(dp: int, dt: float):
    """Exact zero-order-hold double integrator, state [p; v], input acceleration."""
    I = np.eye(dp)
    Z = np.zeros((dp, dp))
    A = np.block([[I, dt * I], [Z, I]])
    B = np.vstack([0.5 * dt * dt * I, dt * I])
    return A, B


def pair_list(N: int) -> np.ndarray:
    """Dense all-pairs list (i < j) in lexicographic order, shape [P, 2]."""
    if N < 2:
        return np.zeros((0, 2), dtype=np.int32)
    i, j = np.triu_indices(N, k=1)
    return np.stack([i, j], axis=1).astype(np.int32)


@dataclasses.dataclass
class Batch:
    nx: int
    nu: int
    dp: int
    N: np.ndarray
    T: np.ndarray
    A: np.ndarray
    B: np.ndarray
    umin: np.ndarray
    umax: np.ndarray
    Qd: np.ndarray
    Rd: np.ndarray
    Qfd: np.ndarray
    x_init: np.ndarray
    x_ref: np.ndarray
    a: np.ndarray
    w0: np.ndarray
    d_min: np.ndarray
    rho: np.ndarray
    targets: Optional[np.ndarray] = None
    meta: dict = dataclasses.field(default_factory=dict)
    # coupled pairs: None = all pairs of every scenario (lexicographic); else
    # pair_count [n_scen] and pair_ij [sum pair_count, 2] (i < j), and the
    # pair-step rows of `a` follow this list
    pair_count: Optional[np.ndarray] = None
    pair_ij: Optional[np.ndarray] = None
    # heterogeneous agents: per-agent dynamics A_agent [sum N, nx, nx] and
    # B_agent [sum N, nx, nu]; None = every agent has the shared A, B
    A_agent: Optional[np.ndarray] = None
    B_agent: Optional[np.ndarray] = None

    @property
    def n_scen(self) -> int:
        return int(self.N.shape[0])

    @property
    def P(self) -> np.ndarray:
        if self.pair_count is not None:
            return self.pair_count.astype(np.int64)
        return (self.N.astype(np.int64) * (self.N - 1)) // 2

    @property
    def pair_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.P)])

    def pairs_of(self, k: int) -> np.ndarray:
        """[P_k, 2] coupled pairs of scenario k."""
        if self.pair_ij is None:
            return pair_list(int(self.N[k]))
        po = self.pair_off
        return self.pair_ij[po[k]:po[k + 1]]

    @property
    def agent_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N.astype(np.int64))])

    @property
    def pairstep_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.P * self.T)])

    @property
    def agentstep_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N.astype(np.int64) * self.T)])

    def scenario(self, k: int) -> "Batch":
        return self.subset([k])

    def subset(self, idx: Sequence[int]) -> "Batch":
        ao, po, so = self.agent_off, self.pairstep_off, self.agentstep_off
        cat = lambda arr, off: np.concatenate([arr[off[k]:off[k + 1]] for k in idx]) if len(idx) else arr[:0]
        return Batch(
            nx=self.nx, nu=self.nu, dp=self.dp,
            N=self.N[list(idx)].copy(), T=self.T[list(idx)].copy(),
            A=self.A, B=self.B, umin=self.umin, umax=self.umax,
            Qd=cat(self.Qd, ao), Rd=cat(self.Rd, ao), Qfd=cat(self.Qfd, ao),
            x_init=cat(self.x_init, ao), x_ref=cat(self.x_ref, ao),
            a=cat(self.a, po), w0=cat(self.w0, so),
            d_min=self.d_min[list(idx)].copy(), rho=self.rho[list(idx)].copy(),
            targets=None if self.targets is None else cat(self.targets, so),
            meta=dict(self.meta),
            pair_count=None if self.pair_count is None else self.pair_count[list(idx)].copy(),
            pair_ij=None if self.pair_ij is None else cat(self.pair_ij, self.pair_off),
            A_agent=None if self.A_agent is None else cat(self.A_agent, ao),
            B_agent=None if self.B_agent is None else cat(self.B_agent, ao),
        )

    def contiguous(self) -> "Batch":
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, np.ndarray):
                setattr(self, f.name, np.ascontiguousarray(v))
        return self


def _draw_separated(rng: SplitMix64, n: int, dp: int, lo: float, hi: float, sep: float) -> np.ndarray:
    pts: List[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        c = lo + (hi - lo) * rng.uniform(dp)
        tries += 1
        if tries > 1000000:
            raise RuntimeError("cannot place starts with the requested separation")
        if pts:
            d = np.linalg.norm(np.asarray(pts) - c, axis=1)
            if d.min() < sep:
                continue
        pts.append(c)
    return np.asarray(pts)


def _permutation(rng: SplitMix64, n: int) -> np.ndarray:
    perm = np.arange(n)
    for k in range(n - 1, 0, -1):
        j = int(rng.uniform(1)[0] * (k + 1))
        perm[k], perm[j] = perm[j], perm[k]
    return perm


def _min_pair_distance(g: np.ndarray) -> float:
    """g: [N, T, dp]; minimum over i<j and t of ||g_it - g_jt||."""
    N = g.shape[0]
    if N < 2:
        return math.inf
    diff = g[:, None, :, :] - g[None, :, :, :]
    d = np.sqrt((diff ** 2).sum(-1))
    iu = np.triu_indices(N, 1)
    return float(d[iu].min())


def _guess_lines(starts, goals, T, c):
    tt = (np.arange(1, T + 1) / T)[None, :, None]
    return starts[:, None, :] + c * tt * (goals - starts)[:, None, :]


def build_scenario(starts: np.ndarray, goals: np.ndarray, T: int, dt: float, d_min: float,
                   literal: bool = False):
    """Guesses, initial states, halfspace normals for one scenario."""
    N, dp = starts.shape
    if literal:
        c = 1.0
        g = _guess_lines(starts, goals, T, 1.0)
        v0 = np.zeros_like(starts)
    else:
        cands = [2.0 ** -k for k in range(21)] + [0.0]
        c = 0.0
        for cand in cands:
            g = _guess_lines(starts, goals, T, cand)
            if _min_pair_distance(g) >= 1.1 * d_min:
                c = cand
                break
        g = _guess_lines(starts, goals, T, c)
        v0 = c * (goals - starts) / (T * dt)
    x_init = np.concatenate([starts, v0], axis=1)
    x_ref = np.concatenate([goals, np.zeros_like(goals)], axis=1)
    pl = pair_list(N)
    if len(pl):
        diff = g[pl[:, 0]] - g[pl[:, 1]]              # [P, T, dp]
        nrm = np.linalg.norm(diff, axis=-1, keepdims=True)
        a = (diff / nrm).reshape(-1, dp)
    else:
        a = np.zeros((0, dp))
    w0 = g.reshape(-1, dp)
    return x_init, x_ref, a, w0, c


def nearest_neighbour_pairs(batch: Batch, k: int) -> Batch:
    """Sparse coupling: each agent keeps the pairs to its k nearest agents at
    t = 0 (the union over both ends, i < j, lexicographic), the rest of the
    instance unchanged (the normals of the kept pairs are the dense ones)."""
    counts, lists, a_rows = [], [], []
    po = batch.pairstep_off
    for s in range(batch.n_scen):
        N, T = int(batch.N[s]), int(batch.T[s])
        x0 = batch.x_init[batch.agent_off[s]:batch.agent_off[s + 1], :batch.dp]
        keep = np.zeros((N, N), dtype=bool)
        if N > 1:
            d = np.sqrt(((x0[:, None, :] - x0[None, :, :]) ** 2).sum(-1))
            np.fill_diagonal(d, np.inf)
            for i in range(N):
                for j in np.argsort(d[i], kind="stable")[:min(k, N - 1)]:
                    keep[min(i, int(j)), max(i, int(j))] = True
        dense = pair_list(N)
        sel = np.array([keep[i, j] for i, j in dense], dtype=bool) if len(dense) else np.zeros(0, dtype=bool)
        lists.append(dense[sel])
        counts.append(int(sel.sum()))
        a_s = batch.a[po[s]:po[s + 1]].reshape(len(dense), T, batch.dp) if len(dense) else np.zeros((0, T, batch.dp))
        a_rows.append(a_s[sel].reshape(-1, batch.dp))
    return dataclasses.replace(batch, a=np.concatenate(a_rows) if a_rows else batch.a[:0],
                               pair_count=np.asarray(counts, dtype=np.int32),
                               pair_ij=(np.concatenate(lists).astype(np.int32) if lists else
                                        np.zeros((0, 2), dtype=np.int32)))


def heterogeneous_agents(batch: Batch, seed: int, damping=(0.0, 0.5), mass=(0.8, 1.25)) -> Batch:
    """Mixed models: agent i of the batch gets velocity damping c_i and mass m_i
    (seeded, uniform in the given ranges) on the batch's double integrator,
    v_{t+1} = (1 - c_i dt) v_t + (dt / m_i) u_t and p_{t+1} = p_t + dt v_t +
    (dt^2 / 2m_i) u_t; everything else (costs, guesses, normals) unchanged."""
    rng = np.random.default_rng(seed)
    na = int(batch.N.sum())
    dp, nx = batch.dp, batch.nx
    dt = float(batch.A[0, dp])
    c = rng.uniform(damping[0], damping[1], na)
    m = rng.uniform(mass[0], mass[1], na)
    I = np.eye(dp)
    A = np.zeros((na, nx, nx))
    B = np.zeros((na, nx, dp))
    for i in range(na):
        A[i, :dp, :dp] = I
        A[i, :dp, dp:] = dt * I
        A[i, dp:, dp:] = (1.0 - c[i] * dt) * I
        B[i, :dp] = 0.5 * dt * dt / m[i] * I
        B[i, dp:] = dt / m[i] * I
    return dataclasses.replace(batch, A_agent=A, B_agent=B)


WORKLOADS = {"pair": 1, "ring14": 2, "mixed": 3, "swarm3d": 4, "diff": 5}

_DEFAULTS = {
    1: dict(dp=2, n_scen=1),
    2: dict(dp=2, n_scen=1),
    3: dict(dp=2, n_scen=4096),
    4: dict(dp=3, n_scen=1),
    5: dict(dp=2, n_scen=64),
}


def _model(dp: int, dt: float, umax: float, q_pos=1.0, q_vel=0.1, r=0.1, qf_scale=10.0):
    A, B = double_integrator(dp, dt)
    nx, nu = 2 * dp, dp
    Qd = np.concatenate([np.full(dp, q_pos), np.full(dp, q_vel)])
    Rd = np.full(nu, r)
    Qfd = qf_scale * Qd
    umin = np.full(nu, -umax)
    umaxv = np.full(nu, umax)
    return A, B, Qd, Rd, Qfd, umin, umaxv


def _scenario_points(cfg: int, k: int, rng: SplitMix64, dp: int, N_override=None, T_override=None):
    if cfg in (1, 2):
        N = 2 if cfg == 1 else 14
        T = 20
        sigma = 0.05 if cfg == 1 else 0.1
        phi = 2.0 * math.pi * np.arange(N) / N
        ring = 5.0 * np.stack([np.cos(phi), np.sin(phi)], axis=1)
        if N_override is not None:
            N = N_override
            phi = 2.0 * math.pi * np.arange(N) / N
            ring = 5.0 * np.stack([np.cos(phi), np.sin(phi)], axis=1)
        if T_override is not None:
            T = T_override
        starts = ring + sigma * rng.normal(N * 2).reshape(N, 2)
        goals = -ring + sigma * rng.normal(N * 2).reshape(N, 2)
        return N, T, starts, goals, 0.5, 1.0, 1.0
    if cfg in (3, 5):
        if cfg == 3:
            N = rng.randint(2, 32)
            T = rng.randint(20, 40)
        else:
            N, T = 16, 30
        if N_override is not None:
            N = N_override
        if T_override is not None:
            T = T_override
        d = 0.4
        starts = _draw_separated(rng, N, 2, -5.0, 5.0, 2 * d)
        goals = starts[_permutation(rng, N)]
        return N, T, starts, goals, d, 1.0, 1.0
    if cfg == 4:
        N = 512 if N_override is None else N_override
        T = 40 if T_override is None else T_override
        d = 0.5
        starts = _draw_separated(rng, N, 3, -20.0, 20.0, 2 * d)
        goals = -starts
        return N, T, starts, goals, d, 2.0, 2.0
    raise ValueError(f"unknown config {cfg}")


def make_workload(name: str, n_scen: Optional[int] = None, literal: bool = False,
                  N_override: Optional[int] = None, T_override: Optional[int] = None,
                  dt: float = 0.1, first: int = 0) -> Batch:
    """Instances of the named synthetic workload ("pair", "ring14", "mixed",
    "swarm3d", "diff"), seeded per scenario; scenario ids first .. first+n_scen-1."""
    cfg = WORKLOADS[name]
    dp = _DEFAULTS[cfg]["dp"]
    S = _DEFAULTS[cfg]["n_scen"] if n_scen is None else n_scen
    scen = []
    for k in range(first, first + S):
        rng = SplitMix64((cfg << 32) + k)
        N, T, starts, goals, d, rho, umax = _scenario_points(cfg, k, rng, dp, N_override, T_override)
        x_init, x_ref, a, w0, c = build_scenario(starts, goals, T, dt, d, literal=literal)
        targets = None
        if cfg == 5:
            targets = -5.0 + 10.0 * rng.uniform(N * T * 2).reshape(N * T, 2)
        scen.append(dict(N=N, T=T, x_init=x_init, x_ref=x_ref, a=a, w0=w0, d=d, rho=rho,
                         umax=umax, c=c, targets=targets))
    umax = scen[0]["umax"]
    return make_batch(scen, dp=dp, dt=dt, umax=umax, meta=dict(workload=name, literal=literal))


def make_batch(scen: List[dict], dp: int, dt: float, umax: float, meta: Optional[dict] = None,
               q_pos=1.0, q_vel=0.1, r=0.1, qf_scale=10.0) -> Batch:
    """Pack per-scenario dictionaries (N, T, x_init, x_ref, a, w0, d, rho[, targets])."""
    A, B, Qd, Rd, Qfd, umin, umaxv = _model(dp, dt, umax, q_pos, q_vel, r, qf_scale)
    Ns = np.array([s["N"] for s in scen], dtype=np.int32)
    Ts = np.array([s["T"] for s in scen], dtype=np.int32)
    tot = int(Ns.sum())
    nx, nu = 2 * dp, dp
    tg = [s.get("targets") for s in scen]
    b = Batch(
        nx=nx, nu=nu, dp=dp, N=Ns, T=Ts, A=A, B=B, umin=umin, umax=umaxv,
        Qd=np.tile(Qd, (tot, 1)), Rd=np.tile(Rd, (tot, 1)), Qfd=np.tile(Qfd, (tot, 1)),
        x_init=np.concatenate([s["x_init"] for s in scen]).reshape(tot, nx),
        x_ref=np.concatenate([s["x_ref"] for s in scen]).reshape(tot, nx),
        a=np.concatenate([s["a"] for s in scen]).reshape(-1, dp),
        w0=np.concatenate([s["w0"] for s in scen]).reshape(-1, dp),
        d_min=np.array([s["d"] for s in scen], dtype=np.float64),
        rho=np.array([s["rho"] for s in scen], dtype=np.float64),
        targets=None if any(t is None for t in tg) else np.concatenate(tg).reshape(-1, dp),
        meta=dict(meta or {}, c=[s.get("c") for s in scen], dt=dt),
    )
    return b.contiguous()


def random_scenario(seed: int, N: int, T: int, dp: int = 2, box: float = 5.0, d_min: float = 0.4,
                    rho: float = 1.0, umax: float = 1.0, dt: float = 0.1, literal: bool = False) -> Batch:
    """One scenario with N agents: starts in a box, goals a permutation of starts."""
    rng = SplitMix64((7 << 32) + seed)
    starts = _draw_separated(rng, N, dp, -box, box, 2 * d_min)
    goals = starts[_permutation(rng, N)] if N > 1 else -starts
    x_init, x_ref, a, w0, c = build_scenario(starts, goals, T, dt, d_min, literal=literal)
    return make_batch([dict(N=N, T=T, x_init=x_init, x_ref=x_ref, a=a, w0=w0, d=d_min, rho=rho,
                            umax=umax, c=c)], dp=dp, dt=dt, umax=umax, meta=dict(seed=seed))
