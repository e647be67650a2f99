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
    approaches the paper's from above as R grows (R = 15 against R = 10).
  - Frame: the net body force (rho - rho^B0) g of a periodic column drives
    the liquid upwards; its volume mean rises at 0.10 U_th in both channels
    (measured 0.103 and 0.111), so relative to the liquid the clean bubble
    rises at 0.70 (2R/L_x = 0.4) and 1.01 (0.2) U_th: the drift explains a
    tenth of U_th of the excess over the paper's values, not all of it.
  - The Eo = 10 Bi sweep at 2R/L_x = 0.4 (Sec. 3.4's trends): surfactant
    lowers the terminal Re below the clean bubble's, Re grows with Bi, and
    the interface's psi_min grows and psi_max falls with Bi (measured Re
    5.968 clean, 5.598 / 5.655 / 5.790 at Bi = 0.5 / 1 / 10; psi_min 1.088 /
    1.329 / 1.762, psi_max 3.334 / 3.159 / 2.738)."""
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


class History(np.ndarray):
    """U_z / U_th every 500 steps; .liquid: the liquid's volume-mean u_z /
    U_th at the end; .diag: the last diagnostics; .re: Re every 500 steps."""


def _history(R, shape, surfactant, steps, Eo=1.0, Bi=10.0):
    cfg = W.bubble_rise_3d(R, shape, Eo=Eo, surfactant=surfactant, Bi=Bi)
    f = W.initial_fields(cfg)
    s = solver(cfg, "f32")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    uth = W.bubble_rise_uth(cfg)
    u, re, done = [], [], 0
    for t in range(500, steps + 1, 500):
        s.step(t - done)
        done = t
        d = s.diagnostics()
        u.append(d["U"][2] / uth)
        re.append(d["Re"])
    fl = s.fields()
    s.close()
    h = np.array(u).view(History)
    h.liquid = float(fl["u"][2][fl["phi"] < 0].mean()) / uth
    h.diag = d
    h.re = np.array(re)
    return h


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


def test_resolution_trend_towards_the_paper(runs, printed):
    r10, r15 = terminal(runs["clean04"]), terminal(runs["clean04_R15"])
    assert printed["bubble_clean_2R/Lx=0.4"] < r15 < r10, (r10, r15)


def test_liquid_drift_and_relative_velocity(runs):
    """Relative to the liquid's volume-mean velocity (driven upwards by the
    net body force of the periodic column) the bubble is slower than in the
    lab frame by the drift, and the wider channel still rises faster."""
    c04, c02 = runs["clean04"], runs["clean02"]
    for h in (c04, c02):
        assert 0.05 < h.liquid < 0.15, h.liquid
    rel04, rel02 = terminal(c04) - c04.liquid, terminal(c02) - c02.liquid
    assert rel04 < rel02, (rel04, rel02)
    # measured 0.70 and 1.01 (lab frame 0.81 and 1.12)
    assert 0.6 < rel04 < 0.8 and 0.9 < rel02 < 1.1, (rel04, rel02)


@pytest.fixture(scope="module")
def bi_sweep():
    out = {"clean": _history(10, (5, 5, 10), False, 16000, Eo=10.0)}
    for bi in (0.5, 1.0, 10.0):
        out[bi] = _history(10, (5, 5, 10), True, 16000, Eo=10.0, Bi=bi)
    return out


def test_eo10_bi_sweep_trends(bi_sweep):
    """Sec. 3.4 at Eo = 10, 2R/L_x = 0.4: surfactant retards the bubble (Re
    below the clean bubble's), the retardation weakens as Bi grows (Re rises
    with Bi), and faster exchange with the bulk evens the interface's
    surfactant out (psi_min rises, psi_max falls with Bi)."""
    def term_re(h):
        return float(h.re[-len(h.re) // 4:].mean())
    re_clean = term_re(bi_sweep["clean"])
    bis = (0.5, 1.0, 10.0)
    re = [term_re(bi_sweep[b]) for b in bis]
    pmin = [bi_sweep[b].diag["psi_min"] for b in bis]
    pmax = [bi_sweep[b].diag["psi_max"] for b in bis]
    assert max(re) < re_clean, (re, re_clean)
    assert re[0] < re[1] < re[2], re
    assert pmin[0] < pmin[1] < pmin[2], pmin
    assert pmax[0] > pmax[1] > pmax[2], pmax
