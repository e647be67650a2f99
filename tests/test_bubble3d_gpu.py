"""The buoyant bubble rise of Sec. 3.4 in 3D (Eo = 1, Mo = 0.1, density and
viscosity ratios 10, walls on x and y, periodic z) on the GPU.

  - Parity: a small channel (R = 4) with soluble surfactant against the
    oracle in FP64.
  - Physics at R = 10 (FP32), measured terminal U/U_th (Eq. 35): clean 0.806
    at 2R/L_x = 0.4 and 1.12 at 0.2; with surfactant 0.724 at 0.4, after an
    early maximum of 0.740.  The paper prints 0.552 / 0.811 (clean) at an
    unstated R.  The test checks what holds at any resolution: the bubble
    rises faster in the wider channel, surfactant retards it after the early
    maximum the paper describes, and at 2R/L_x = 0.4 the clean velocity
    approaches the paper's from above as R grows (R = 15 against R = 10)."""
import numpy as np
import pytest

import workloads as W
from oracle.ora import Oracle

from test_parity_gpu import errors, solver

pytestmark = pytest.mark.gpu


def test_small_bubble_matches_oracle():
    cfg = W.bubble_rise_3d(R=4)
    f = W.initial_fields(cfg, seed=4, noise=0.02, u0=1e-4)
    o = Oracle(cfg)
    o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    s = solver(cfg, "f64")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    o.step(30)
    s.step(30)
    err = errors(o.fields(), s.fields())
    s.close()
    assert max(err.values()) < 1e-9, err


def _history(R, shape, surfactant, steps):
    cfg = W.bubble_rise_3d(R, shape, surfactant=surfactant)
    f = W.initial_fields(cfg)
    s = solver(cfg, "f32")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    uth = W.bubble_rise_uth(cfg)
    u, done = [], 0
    for t in range(500, steps + 1, 500):
        s.step(t - done)
        done = t
        u.append(s.diagnostics()["U"][2] / uth)
    s.close()
    return np.array(u)


@pytest.fixture(scope="module")
def runs():
    return {"clean04": _history(10, (5, 5, 10), False, 16000),
            "surf04": _history(10, (5, 5, 10), True, 16000),
            "clean02": _history(10, (10, 10, 10), False, 16000),
            "clean04_R15": _history(15, (5, 5, 10), False, 20000)}


def terminal(u):
    return float(u[-len(u) // 4:].mean())


def test_confinement_and_retardation(runs):
    c04, s04, c02 = (terminal(runs[k]) for k in ("clean04", "surf04", "clean02"))
    assert 0.5 < c04 < c02, (c04, c02)
    assert s04 < 0.95 * c04, (s04, c04)
    assert runs["surf04"].max() > 1.01 * s04, (runs["surf04"].max(), s04)


def test_resolution_trend_towards_the_paper(runs):
    r10, r15 = terminal(runs["clean04"]), terminal(runs["clean04_R15"])
    assert 0.552 < r15 < r10, (r10, r15)
