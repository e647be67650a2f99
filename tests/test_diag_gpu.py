"""Diagnostics of the CUDA path (lbs_diagnostics, through the C ABI): the
droplet/bubble velocity U of Eqs. 33-34, Re and the aspect ratio of Sec. 3.4,
the centroid, the interface psi statistics and max |u|.  They are the labels
the surrogate learns from, so they are checked twice:

  - on a hand-built state whose values are known in closed form (the same
    state pins the oracle's diagnostics, tests/test_oracle_step_pins.py);
  - against the oracle's diagnostics after a run of the droplet and the
    bubble: FP64 storage to 1e-9; FP32 storage after 300 steps within the
    FP32 field errors (the region rho^N >= 0 is the same cell set when no
    cell's rho^N sits within the FP32 error of 0; the test checks that).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.ora import Oracle

from test_oracle_step_pins import hand_built
from test_parity_gpu import bubble, droplet, run_both, solver

pytestmark = pytest.mark.gpu

KEYS = ("U", "centroid", "aspect_ratio", "Re", "psi_av", "psi_min", "psi_max", "umax",
        "mass_R", "mass_B")


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_gpu_diagnostics_of_a_hand_built_state(D, storage):
    cfg, phi, psi, u, box, vals, (x, y, z) = hand_built(D)
    s = solver(cfg, storage)
    s.init_fields(phi, psi, np.zeros_like(phi), u)
    d = s.diagnostics()
    rtol = 1e-12 if storage == "f64" else 2e-6
    red = phi >= 0
    n = red.sum()
    U = [u[a][red].mean() for a in range(3)]
    for a in range(D):
        assert d["U"][a] == pytest.approx(U[a], rel=rtol, abs=1e-15)
    cen = [x[red].mean(), y[red].mean(), z[red].mean()]
    for a in range(D):
        assert d["centroid"][a] == pytest.approx(cen[a], rel=1e-13)
    sides = [box[2].stop - box[2].start, box[1].stop - box[1].start, box[0].stop - box[0].start]
    vol = int(np.prod(sides[:D]))

    def second(a):
        return vol // sides[a] * sides[a] * (sides[a] ** 2 - 1) / 12.0

    assert d["aspect_ratio"] == pytest.approx(math.sqrt(second(0) / second(D - 1)), rel=1e-12)
    R = math.sqrt(n / math.pi) if D == 2 else (3 * n / (4 * math.pi)) ** (1 / 3)
    assert d["Re"] == pytest.approx(2 * cfg["rhoB0"] * abs(U[D - 1]) * R / cfg["muB0"], rel=rtol)
    assert d["psi_av"] == pytest.approx(np.mean(vals), rel=rtol)
    assert d["psi_min"] == pytest.approx(min(vals), rel=rtol)
    assert d["psi_max"] == pytest.approx(max(vals), rel=rtol)
    assert d["umax"] == pytest.approx(np.sqrt((u ** 2).sum(axis=0)).max(), rel=rtol)
    mR = (cfg["rhoR0"] * 0.5 * (1 + phi)).sum()
    assert d["mass_R"] == pytest.approx(mR, rel=1e-14 if storage == "f64" else 1e-7)
    s.close()


def compare(d_o, d_s, rtol):
    out = {}
    for k in KEYS:
        a = np.atleast_1d(np.asarray(d_o[k], dtype=float))
        b = np.atleast_1d(np.asarray(d_s[k], dtype=float))
        scale = max(np.abs(a).max(), 1e-30)
        out[k] = float(np.abs(a - b).max() / scale)
    bad = {k: v for k, v in out.items() if v > rtol.get(k, rtol["*"])}
    assert not bad, (bad, out)


@pytest.mark.parametrize("make", [droplet, bubble], ids=["droplet", "bubble"])
def test_diagnostics_match_oracle_f64(make):
    cfg = make()
    o, s = run_both(cfg, 60, "f64", u0=1e-3)
    compare(o.diagnostics(), s.diagnostics(), {"*": 1e-9})
    s.close()


@pytest.mark.parametrize("make", [droplet, bubble], ids=["droplet", "bubble"])
def test_diagnostics_match_oracle_f32(make):
    cfg = make()
    o, s = run_both(cfg, 300, "f32")
    ref = o.fields()
    # the indicator rho^N >= 0 and the band |rho^N| < 0.5 select the same
    # cells on both sides when no rho^N lies within the FP32 error of the
    # thresholds
    margin = np.min([np.abs(ref["phi"]).min(), np.abs(np.abs(ref["phi"]) - 0.5).min()])
    assert margin > 1e-4, margin
    # (colour masses: the FP32 rounding of the initial populations, ~1e-7)
    compare(o.diagnostics(), s.diagnostics(), {"*": 1e-4, "mass_R": 3e-7, "mass_B": 3e-7})
    s.close()


def test_bubble_diagnostics_3d_match_oracle_f64():
    """D3Q19 bubble between walls: the same comparison in 3D."""
    c = W.base(22, 40, 19)
    aR, aB = W._alphas(3, 0.1, 1.0)
    c.update(wall=[1, 0, 1], rhoR0=0.1, rhoB0=1.0, alphaR=aR, alphaB=aB, muB0=0.05,
             muR0=0.005, sigma0=0.01, E0=0.5, psi_inf=4.0, Ds=0.05, Db=0.05, rd=1e-3,
             ra=2e-3, source=0, g=[0, -2e-5, 0], R=5.0, C0=0.5, psi0=0.0,
             center=[10.7, 12.3, 8.9])
    o, s = run_both(c, 30, "f64", u0=1e-4)
    compare(o.diagnostics(), s.diagnostics(), {"*": 1e-9})
    s.close()
