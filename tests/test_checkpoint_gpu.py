"""Checkpoint / restart and the error statuses of a single context, through
the C ABI (lbs_save_state, lbs_load_state, lbs_sync).

The time stepping of Sec. 2.2 carries state from step to step (populations,
psi and C, the Adams-Bashforth history S^{t-1}, B^{t-1} of Eqs. 23-24, the
conserved total of the rescale, the step counter).  A restart from a saved
state must reproduce the uninterrupted run bit for bit."""
import numpy as np
import pytest

import workloads as W

from test_parity_gpu import bubble, solver

pytestmark = pytest.mark.gpu


def shear3(nx=34, ny=20, nz=17, R=5.0):
    c = W.shear_droplet_3d(nx=nx, ny=ny, nz=nz, R=R)
    c["center"] = [(nx - 1) / 2 + 0.3, (ny - 1) / 2 - 0.2, (nz - 1) / 2 + 0.1]
    return c


def same(a, b):
    """Every field identical, bit for bit."""
    return all(np.array_equal(a[k], b[k]) for k in ("rho", "u", "phi", "psi", "C"))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_restart_bit_exact_2d(storage):
    """1000 steps of the bubble rise against 500 steps, save, a fresh context
    loading the state, and 500 more steps: identical fields and totals."""
    cfg = bubble()
    f = W.initial_fields(cfg, seed=5, noise=0.02)
    a = solver(cfg, storage)
    a.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    a.step(500)
    state = a.save_state()
    a.step(500)
    b = solver(cfg, storage)
    b.load_state(state)
    assert b.diagnostics()["step"] == 500
    b.step(500)
    da, db = a.diagnostics(), b.diagnostics()
    assert same(a.fields(), b.fields())
    for k in ("mass_R", "mass_B", "surf_total", "surf_pre_rescale", "rescale_factor"):
        assert da[k] == db[k], k
    assert da["step"] == db["step"] == 1000
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_restart_bit_exact_3d(storage):
    """The same on the D3Q19 sheared droplet between moving walls."""
    cfg = shear3()
    f = W.initial_fields(cfg, seed=3, noise=0.02)
    a = solver(cfg, storage)
    a.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    a.step(60)
    state = a.save_state()
    a.step(60)
    b = solver(cfg, storage)
    b.load_state(state)
    b.step(60)
    assert same(a.fields(), b.fields())
    assert a.diagnostics()["surf_total"] == b.diagnostics()["surf_total"]
    a.close()
    b.close()


def test_load_state_refuses_other_grid_and_storage():
    from paper_2311_15242_gb300.lbs import LBS_EINVAL, LbsError
    cfg = bubble()
    f = W.initial_fields(cfg, seed=5)
    a = solver(cfg, "f32")
    a.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    state = a.save_state()
    for other_cfg, st in ((bubble(nx=42), "f32"), (cfg, "f16")):
        b = solver(other_cfg, st)
        with pytest.raises(LbsError) as e:
            b.load_state(state)
        assert e.value.code == LBS_EINVAL
        b.close()
    with pytest.raises(LbsError) as e:
        a.load_state(state[:-1])
    assert e.value.code == LBS_EINVAL
    a.close()


@pytest.mark.parametrize("persistent", [True, False], ids=["one_launch", "graph_loop"])
def test_timeout_then_continue_matches_fresh_context(persistent):
    """A one-poll barrier limit makes the one-launch SOR give up (LBS_ETIMEOUT
    at the next sync).  With the default limit restored and no
    re-initialisation, the context steps on exactly like a fresh context
    loaded with its state: nothing of the interrupted barrier survives into
    the next launch."""
    from paper_2311_15242_gb300.lbs import LBS_ETIMEOUT, LbsError
    cfg = bubble()
    f = W.initial_fields(cfg, seed=9, noise=0.02)
    a = solver(cfg, "f32")
    a.set_sor_tile(5)
    a.set_sor_persistent(persistent)
    a.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    a.step(3)
    a.sync()
    a.set_sor_wait_limit(1)
    codes = []
    for _ in range(4):
        try:
            a.step(1)
            a.sync()
        except LbsError as e:
            codes.append(e.code)
    if persistent:
        assert LBS_ETIMEOUT in codes, codes
    else:
        assert codes == [], codes  # the graph loop has no grid barrier
    a.set_sor_wait_limit(1 << 24)
    state = a.save_state()
    b = solver(cfg, "f32")
    b.set_sor_tile(5)
    b.set_sor_persistent(persistent)
    b.load_state(state)
    for _ in range(3):
        a.step(7)
        b.step(7)
        assert same(a.fields(), b.fields())
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["2d_one_launch", "2d_graph_loop", "3d"])
def test_sor_not_converged_reports_enoconv(case):
    """A solve limited to one sweep (one blocked round in 2D) with a
    tolerance it cannot meet reports LBS_ENOCONV at the next sync; the
    context keeps stepping."""
    from paper_2311_15242_gb300.lbs import LBS_ENOCONV, LbsError
    cfg = shear3() if case == "3d" else bubble()
    cfg = dict(cfg, sor_max_iter=1, sor_tol=1e-12)
    f = W.initial_fields(cfg, seed=2, noise=0.02)
    s = solver(cfg, "f32")
    if case == "2d_graph_loop":
        s.set_sor_persistent(False)
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    s.step(2)
    with pytest.raises(LbsError) as e:
        s.sync()
    assert e.value.code == LBS_ENOCONV
    s.step(1)
    with pytest.raises(LbsError):
        s.sync()
    assert s.diagnostics()["step"] == 3
    s.close()


def test_nan_input_reports_ediverged():
    """A NaN planted on the host in one cell of the initial psi makes the
    conserved total non-finite: the first step reports LBS_EDIVERGED."""
    from paper_2311_15242_gb300.lbs import LBS_EDIVERGED, LbsError
    cfg = bubble()
    f = W.initial_fields(cfg, seed=2)
    psi = np.array(f["psi"], dtype=np.float64, copy=True)
    psi.reshape(-1)[psi.size // 2 + 7] = np.nan
    s = solver(cfg, "f32")
    s.init_fields(f["phi"], psi, f["C"], f["u"])
    s.step(1)
    with pytest.raises(LbsError) as e:
        s.sync()
    assert e.value.code == LBS_EDIVERGED
    s.close()
