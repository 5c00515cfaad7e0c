"""The allocation-free entry point tadmm_solve_noalloc.

It serves callers that must not allocate device memory while they run (for
example a real-time control loop that may only allocate at start-up, or a
program whose device memory belongs to an outside allocator).  This test plays
such a caller: it owns its device input and output buffers, calls the entry
point twice in a row through the C ABI on two different scenarios, and checks
each result against the regular create/solve/get_solution path within the
parity tolerance of the GPU tests (1e-9 relative).  The second call must not
see anything left in the shared static scratch by the first, and after one
warm-up call per model size (which loads the library's kernels) the calls
leave the device's free memory unchanged.
"""
import ctypes as C

import numpy as np
import pytest

from instances import make_workload

pytestmark = pytest.mark.gpu


class ScenarioDev(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nu", C.c_int32), ("dp", C.c_int32), ("N", C.c_int32), ("T", C.c_int32),
                ("A", C.c_void_p), ("B", C.c_void_p), ("umin", C.c_void_p), ("umax", C.c_void_p),
                ("Qd", C.c_void_p), ("Rd", C.c_void_p), ("Qfd", C.c_void_p), ("x_init", C.c_void_p),
                ("x_ref", C.c_void_p), ("a", C.c_void_p), ("w0", C.c_void_p), ("d_min", C.c_double),
                ("rho", C.c_double)]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max())) if a.size else 0.0


class _Call:
    """Caller-owned device buffers for tadmm_solve_noalloc on scenario 0 of `b`
    (allocated up front, as a caller that cannot allocate later would)."""

    def __init__(self, tg, torch, b, tol, max_iter, start_mode=2):
        dev = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
        self.keep = dict(A=dev(b.A), B=dev(b.B), umin=dev(b.umin), umax=dev(b.umax), Qd=dev(b.Qd), Rd=dev(b.Rd),
                         Qfd=dev(b.Qfd), x_init=dev(b.x_init), x_ref=dev(b.x_ref),
                         a=dev(b.a if b.a.size else np.zeros((1, b.dp))), w0=dev(b.w0))
        N, T = int(b.N[0]), int(b.T[0])
        self.N, self.T, self.P, self.b = N, T, N * (N - 1) // 2, b
        self.s = ScenarioDev(b.nx, b.nu, b.dp, N, T, *[self.keep[k].data_ptr() for k in
                                                       ("A", "B", "umin", "umax", "Qd", "Rd", "Qfd", "x_init",
                                                        "x_ref", "a", "w0")],
                             float(b.d_min[0]), float(b.rho[0]))
        self.X = torch.full((N * (T + 1) * b.nx,), np.nan, dtype=torch.float64, device="cuda")
        self.U = torch.full((N * T * b.nu,), np.nan, dtype=torch.float64, device="cuda")
        self.TH = torch.full((max(self.P * T, 1),), np.nan, dtype=torch.float64, device="cuda")
        self.SI = torch.zeros(2, dtype=torch.int32, device="cuda")
        self.RS = torch.zeros(2, dtype=torch.float64, device="cuda")
        self.tol, self.max_iter, self.start_mode = tol, max_iter, start_mode
        self.L = tg.lib()
        self.L.tadmm_solve_noalloc.argtypes = [C.POINTER(ScenarioDev), C.c_int32, C.c_double, C.c_int32,
                                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_void_p]
        self.stream = torch.cuda.current_stream().cuda_stream

    def launch(self):
        rc = self.L.tadmm_solve_noalloc(C.byref(self.s), self.start_mode, self.tol, self.max_iter,
                                        self.X.data_ptr(), self.U.data_ptr(),
                                        self.TH.data_ptr() if self.P else None, self.SI.data_ptr(),
                                        self.RS.data_ptr(), self.stream)
        assert rc == 0, self.L.tadmm_last_error().decode()

    def result(self):
        b, N, T, P = self.b, self.N, self.T, self.P
        return dict(X=self.X.cpu().numpy().reshape(N, T + 1, b.nx), U=self.U.cpu().numpy().reshape(N, T, b.nu),
                    theta=self.TH.cpu().numpy()[:P * T].reshape(P, T), status=int(self.SI[0]),
                    iters=int(self.SI[1]), r=float(self.RS[0]), s=float(self.RS[1]))


def _regular(tg, b, tol, max_iter, start="turbo"):
    s = tg.Solver(b, precision=64, start=start)
    s.solve(tol, max_iter)
    out = s.split(s.solution())[0]
    s.close()
    return out


def _gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_15838_gb300 import build
    build.build()
    import paper_2602_15838_gb300 as tg
    return torch, tg


def _assert_same(got, ref):
    assert got["status"] == ref["status"] and got["iters"] == ref["iters"]
    assert _rel(got["X"], ref["X"]) <= 1e-9
    assert _rel(got["U"], ref["U"]) <= 1e-9
    assert _rel(got["theta"], ref["theta"]) <= 1e-9
    assert abs(got["r"] - ref["r"]) <= 1e-9 and abs(got["s"] - ref["s"]) <= 1e-9


def test_noalloc_matches_regular_path_two_calls_in_a_row():
    torch, tg = _gpu_lib()
    calls = [_Call(tg, torch, make_workload("ring14"), 0.0, 25), _Call(tg, torch, make_workload("pair"), 1e-4, 500)]
    calls[0].launch()                        # warm-up: loads the 2D kernels on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for c in calls:                          # the two calls in a row
        c.launch()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0   # nothing allocated on the device
    for c, (tol, max_iter) in zip(calls, ((0.0, 25), (1e-4, 500))):
        _assert_same(c.result(), _regular(tg, c.b, tol, max_iter))


def test_noalloc_3d_and_cold_start_match_regular_path():
    """The 3D model (nx = 6, nu = 3) of the swarm workload with 4 agents, T = 10,
    and a cold start (BaseADMM) of the 2-agent crossing, each against the
    regular path with the same start."""
    torch, tg = _gpu_lib()
    b3 = make_workload("swarm3d", N_override=4, T_override=10)
    c3 = _Call(tg, torch, b3, 0.0, 12)
    c3.launch()
    torch.cuda.synchronize()
    _assert_same(c3.result(), _regular(tg, b3, 0.0, 12))
    bc = make_workload("pair")
    cc = _Call(tg, torch, bc, 1e-4, 500, start_mode=0)
    cc.launch()
    torch.cuda.synchronize()
    _assert_same(cc.result(), _regular(tg, bc, 1e-4, 500, start="cold"))


@pytest.mark.parametrize("fault", ["umin_gt_umax", "negative_R", "nan_Q", "negative_Qf", "inf_w0"])
def test_noalloc_reports_invalid_input_values(fault):
    """Input values are device memory, so the entry point checks them on the
    device by tadmm_create's rules: a bad value gives status
    TADMM_INVALID_INPUT (4), zero iterations and NaN residuals, and the next
    valid call is solved as usual."""
    torch, tg = _gpu_lib()
    b = make_workload("pair")
    bad = b.subset([0])
    if fault == "umin_gt_umax":
        bad.umin = bad.umax + 0.5
    elif fault == "negative_R":
        bad.Rd = bad.Rd.copy(); bad.Rd[1, 0] = -0.1
    elif fault == "nan_Q":
        bad.Qd = bad.Qd.copy(); bad.Qd[0, 2] = np.nan
    elif fault == "negative_Qf":
        bad.Qfd = bad.Qfd.copy(); bad.Qfd[1, 3] = -1.0
    else:
        bad.w0 = bad.w0.copy(); bad.w0[5, 1] = np.inf
    c = _Call(tg, torch, bad, 1e-4, 50)
    c.launch()
    torch.cuda.synchronize()
    r = c.result()
    assert r["status"] == 4 and r["iters"] == 0
    assert np.isnan(r["r"]) and np.isnan(r["s"])
    good = _Call(tg, torch, b, 1e-4, 500)
    good.launch()
    torch.cuda.synchronize()
    _assert_same(good.result(), _regular(tg, b, 1e-4, 500))


def test_noalloc_rejects_oversized_scenario():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15838_gb300 as tg
    L = tg.lib()
    L.tadmm_solve_noalloc.argtypes = [C.POINTER(ScenarioDev), C.c_int32, C.c_double, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = z.data_ptr()
    s = ScenarioDev(4, 2, 2, 2000, 40, p, p, p, p, p, p, p, p, p, p, p, 0.5, 1.0)
    rc = L.tadmm_solve_noalloc(C.byref(s), 2, 1e-4, 10, None, None, None, None, None, None)
    assert rc == tg.EINVAL
    assert "static scratch" in L.tadmm_last_error().decode()
