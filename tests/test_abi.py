"""The C-ABI library builds for sm_103a, loads, exports every symbol declared in
include/tadmm.h, and rejects invalid inputs on the host before any launch
(no GPU needed for these calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libtadmm():
    from paper_2602_15838_gb300 import build
    path = build.build()
    import paper_2602_15838_gb300 as tg
    return tg, tg.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tadmm_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(libtadmm):
    _, L = libtadmm
    names = _declared()
    assert "tadmm_create" in names and "tadmm_solve" in names
    for n in names:
        assert hasattr(L, n), n


def test_version_and_last_error(libtadmm):
    tg, L = libtadmm
    assert b"sm_103a" in L.tadmm_version()
    assert isinstance(L.tadmm_last_error(), bytes)


def _create_rc(tg, batch, **opt):
    hb = tg._HostBatch(batch)
    if opt.get("null_B_agent"):
        hb.s.B_agent = None
    ae, am, at = opt.get("adapt", (0, 10.0, 2.0))
    o = tg.TadmmOptions(opt.get("precision", 64), opt.get("start", 2), 0, 0.0, opt.get("mode", 0), 0, 0, 0,
                        opt.get("flags", 0), ae, am, at, opt.get("relax", 0.0))
    h = C.c_void_p()
    rc = tg.lib().tadmm_create(C.byref(hb.s), C.byref(o), C.byref(h))
    return rc, tg.lib().tadmm_last_error().decode()


@pytest.mark.parametrize("fault", ["nan_q", "neg_r", "box", "rho", "dims", "N0", "prec", "adapt_mode", "adapt_mu",
                                   "pair_dup", "pair_order", "relax_range", "relax_mode", "relax_flags",
                                   "hetero_half", "hetero_nan", "hetero_df64", "homotopy_batched", "homotopy_df64",
                                   "start_range"])
def test_invalid_inputs_rejected_on_host(libtadmm, fault):
    tg, _ = libtadmm
    from instances import make_workload
    b = make_workload("pair")
    opt = {}
    if fault == "nan_q":
        b.Qd = b.Qd.copy(); b.Qd[0, 1] = np.nan
    elif fault == "neg_r":
        b.Rd = b.Rd.copy(); b.Rd[1, 0] = -0.1
    elif fault == "box":
        b.umin = np.array([0.5, -1.0]); b.umax = np.array([0.4, 1.0])
    elif fault == "rho":
        b.rho = np.array([0.0])
    elif fault == "dims":
        b.dp = 3
    elif fault == "N0":
        b.N = np.array([0], dtype=np.int32)
    elif fault == "prec":
        opt["precision"] = 16
    elif fault == "adapt_mode":   # residual balancing runs in the batched mode only
        opt["mode"] = 1
        opt["adapt"] = (5, 10.0, 2.0)
    elif fault == "adapt_mu":
        opt["adapt"] = (5, 1.0, 2.0)
    elif fault in ("hetero_half", "hetero_nan", "hetero_df64"):   # per-agent dynamics
        from instances import heterogeneous_agents
        b = heterogeneous_agents(b, seed=1)
        if fault == "hetero_half":
            opt["null_B_agent"] = True
        elif fault == "hetero_nan":
            b.A_agent[1, 0, 0] = np.nan
        else:
            opt["flags"] = 8
    elif fault == "homotopy_batched":   # the homotopy hot start runs in the plain and graph modes
        opt["start"] = 3
    elif fault == "homotopy_df64":
        opt["start"] = 3
        opt["mode"] = 1
        opt["flags"] = 8
    elif fault == "start_range":
        opt["start"] = 4
    elif fault == "relax_range":   # over-relaxation factor in (0, 2)
        opt["relax"] = 2.0
    elif fault == "relax_mode":    # over-relaxation runs in the batched mode only
        opt["mode"] = 1
        opt["relax"] = 1.5
    elif fault == "relax_flags":   # ... on the group path
        opt["flags"] = 4
        opt["relax"] = 1.5
    elif fault in ("pair_dup", "pair_order"):   # listed pairs: each once, i < j < N
        import dataclasses
        b = make_workload("ring14")
        pl = np.array([[0, 1], [0, 1]] if fault == "pair_dup" else [[1, 0], [2, 3]], dtype=np.int32)
        b = dataclasses.replace(b, pair_count=np.array([2], dtype=np.int32), pair_ij=pl,
                                a=b.a[:2 * int(b.T[0])])
    rc, msg = _create_rc(tg, b, **opt)
    assert rc == tg.EINVAL, msg
    assert msg


def test_null_batch_rejected(libtadmm):
    tg, L = libtadmm
    h = C.c_void_p()
    assert L.tadmm_create(None, None, C.byref(h)) == tg.EINVAL
    assert L.tadmm_solve(None, 1e-4, 10, None) == tg.EINVAL


def test_scenario_over_the_32_bit_index_limit_rejected(libtadmm):
    """A scenario whose per-stage arrays would exceed 2^31 elements (here
    N = 32767 agents, T = 1000) is refused on the host before any of its data is
    read beyond the per-scenario scalars."""
    tg, L = libtadmm
    one = np.ones(64)
    keep = [one]
    dp_ = one.ctypes.data_as(C.POINTER(C.c_double))
    N = np.array([32767], dtype=np.int32)
    T = np.array([1000], dtype=np.int32)
    keep += [N, T]
    i32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    bs = tg.TadmmBatch(1, 4, 2, 2, i32(N), i32(T), dp_, dp_, dp_, dp_, dp_, dp_, dp_, dp_, dp_, dp_, dp_,
                       dp_, dp_, None, None, None, None)
    o = tg.TadmmOptions(64, 2, 0, 0.0, 0, 0, 0, 0, 0, 0, 10.0, 2.0, 0.0)
    h = C.c_void_p()
    assert L.tadmm_create(C.byref(bs), C.byref(o), C.byref(h)) == tg.EINVAL
    assert b"2^31" in L.tadmm_last_error()
