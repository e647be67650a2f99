"""The adsorption test of Sec. 3.1 in 3D (one octant of a droplet between
mirror planes, Eqs. 29-30) on the GPU.

  - Parity: a small octant (R = 4, 20^3 cells) against the oracle in FP64.
  - Physics: at R = 20 and R = 30 (5R cubes, FP32), the interface coverage
    psi/psi_inf (mean over the shell |rhoN| < 0.1) against Eq. 30 and the bulk
    concentration C/C0 along the x axis against Eq. 29 (the sharp-interface
    solutions; readings in workloads.adsorption_analytic), at tau = D t / R^2
    = 0.11, 0.56 and 1.11, the range over which the paper finds them valid.
    The diffuse interface adsorbs over a slightly larger radius than R, so
    psi runs above Eq. 30 (measured: +19 / +14 / +12 % at R = 20, +13 / +9 /
    +8 % at R = 30) and C below Eq. 29 near the interface; both errors shrink
    as R grows, which the test checks alongside bounds above the measured
    values."""
import numpy as np
import pytest

import workloads as W
from oracle.ora import Oracle

from test_parity_gpu import errors, solver

pytestmark = pytest.mark.gpu

TAUS = (0.11, 0.56, 1.11)


def test_small_octant_matches_oracle():
    cfg = W.adsorption_octant_3d(R=4)
    cfg["C0"] = 0.5  # (larger uptake: every term of the source path acts)
    f = W.initial_fields(cfg, seed=5, noise=0.02, u0=1e-4)
    o = Oracle(cfg)
    o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    s = solver(cfg, "f64")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    o.step(30)
    s.step(30)
    err = errors(o.fields(), s.fields())
    s.close()
    assert max(err.values()) < 1e-9, err


def _run(R):
    cfg = W.adsorption_octant_3d(R=R)
    f = W.initial_fields(cfg)
    s = solver(cfg, "f32")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    n = cfg["nx"]
    r = np.sqrt((np.arange(n) + 0.5) ** 2 + 0.5)  # cells (x, 0, 0)
    out, done = [], 0
    for tau in TAUS:
        t = int(round(tau * R * R / cfg["Db"]))
        s.step(t - done)
        done = t
        F = s.fields()
        psi = F["psi"][np.abs(F["phi"]) < 0.1].mean() / cfg["psi_inf"]
        c_an, psi_an = W.adsorption_analytic(cfg, t, r)
        pick = [int(round(R * q - 0.5)) for q in (2.0, 3.0)]
        out.append(dict(psi=psi, psi_an=psi_an, c=F["C"][0, 0, pick] / cfg["C0"],
                        c_an=c_an[pick]))
    s.close()
    return out


@pytest.fixture(scope="module")
def runs():
    return {R: _run(R) for R in (20, 30)}


def test_interface_coverage_against_eq30(runs):
    for R, bound in ((20, 0.22), (30, 0.16)):
        for k, o in enumerate(runs[R]):
            rel = o["psi"] / o["psi_an"] - 1
            assert 0 < rel <= bound, (R, TAUS[k], o["psi"], o["psi_an"])
    for k in range(len(TAUS)):  # converging with the resolution
        e20 = abs(runs[20][k]["psi"] / runs[20][k]["psi_an"] - 1)
        e30 = abs(runs[30][k]["psi"] / runs[30][k]["psi_an"] - 1)
        assert e30 < e20, (TAUS[k], e20, e30)


def test_bulk_profile_against_eq29(runs):
    for R, bound in ((20, 0.045), (30, 0.03)):
        for k, o in enumerate(runs[R]):
            d = np.abs(o["c"] - o["c_an"])
            assert d.max() <= bound, (R, TAUS[k], o["c"], o["c_an"])
    for k in range(len(TAUS)):
        e20 = abs(runs[20][k]["c"][0] - runs[20][k]["c_an"][0])
        e30 = abs(runs[30][k]["c"][0] - runs[30][k]["c_an"][0])
        assert e30 <= e20 + 1e-3, (TAUS[k], e20, e30)
