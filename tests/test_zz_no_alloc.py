"""The allocation-free entry point tadmm_solve_noalloc.

It serves callers that must not allocate device memory while they run (for
example a real-time control loop that may only allocate at start-up, or a
program whose device memory belongs to an outside allocator).  This test plays
such a caller: it owns its device input and output buffers, calls the entry
point twice in a row through the C ABI on two different scenarios, and checks
each result against the regular create/solve/get_solution path within the
parity tolerance of the GPU tests (1e-9 relative).  The second call must not
see anything left in the shared static scratch by the first.
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


def _noalloc_call(tg, torch, b, tol, max_iter):
    """Runs tadmm_solve_noalloc on scenario 0 of `b` with caller-owned device buffers."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    keep = dict(A=dev(b.A), B=dev(b.B), umin=dev(b.umin), umax=dev(b.umax), Qd=dev(b.Qd), Rd=dev(b.Rd),
                Qfd=dev(b.Qfd), x_init=dev(b.x_init), x_ref=dev(b.x_ref),
                a=dev(b.a if b.a.size else np.zeros((1, b.dp))), w0=dev(b.w0))
    N, T = int(b.N[0]), int(b.T[0])
    P = N * (N - 1) // 2
    s = ScenarioDev(b.nx, b.nu, b.dp, N, T, *[keep[k].data_ptr() for k in
                                               ("A", "B", "umin", "umax", "Qd", "Rd", "Qfd", "x_init", "x_ref",
                                                "a", "w0")],
                    float(b.d_min[0]), float(b.rho[0]))
    X = torch.full((N * (T + 1) * b.nx,), np.nan, dtype=torch.float64, device="cuda")
    U = torch.full((N * T * b.nu,), np.nan, dtype=torch.float64, device="cuda")
    TH = torch.full((max(P * T, 1),), np.nan, dtype=torch.float64, device="cuda")
    SI = torch.zeros(2, dtype=torch.int32, device="cuda")
    RS = torch.zeros(2, dtype=torch.float64, device="cuda")
    L = tg.lib()
    L.tadmm_solve_noalloc.argtypes = [C.POINTER(ScenarioDev), C.c_int32, C.c_double, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.tadmm_solve_noalloc(C.byref(s), 2, tol, max_iter, X.data_ptr(), U.data_ptr(),
                               TH.data_ptr() if P else None, SI.data_ptr(), RS.data_ptr(), stream)
    assert rc == 0, L.tadmm_last_error().decode()
    torch.cuda.synchronize()
    return dict(X=X.cpu().numpy().reshape(N, T + 1, b.nx), U=U.cpu().numpy().reshape(N, T, b.nu),
                theta=TH.cpu().numpy()[:P * T].reshape(P, T), status=int(SI[0]), iters=int(SI[1]),
                r=float(RS[0]), s=float(RS[1]))


def _regular(tg, b, tol, max_iter):
    s = tg.Solver(b, precision=64, start="turbo")
    s.solve(tol, max_iter)
    out = s.split(s.solution())[0]
    s.close()
    return out


def test_noalloc_matches_regular_path_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_15838_gb300 import build
    build.build()
    import paper_2602_15838_gb300 as tg

    cases = [(make_workload("ring14"), 0.0, 25), (make_workload("pair"), 1e-4, 500)]
    for b, tol, max_iter in cases:
        got = _noalloc_call(tg, torch, b, tol, max_iter)
        ref = _regular(tg, b, tol, max_iter)
        assert got["status"] == ref["status"] and got["iters"] == ref["iters"]
        assert _rel(got["X"], ref["X"]) <= 1e-9
        assert _rel(got["U"], ref["U"]) <= 1e-9
        assert _rel(got["theta"], ref["theta"]) <= 1e-9
        assert abs(got["r"] - ref["r"]) <= 1e-9 and abs(got["s"] - ref["s"]) <= 1e-9


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
