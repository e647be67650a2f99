"""Shifted 16-bit population storage (FP16 and bfloat16, FP32 arithmetic,
FP64 totals) against the FP64 oracle after 1000 steps.

Every stored moving population is a small number (the total minus a rest
state, or the cell's minority colour); FP16 values are kept scaled by 2^14.
The rest populations are kept in FP32 and absorb the rounding of the moving
ones, rounded without bias, so every cell's colour masses are those of the
FP32 arithmetic.  The
bounds below are the stated per-field accuracy of these forms (about three
times the measured errors), not the FP32 tolerances: FP16 has an 11-bit and
bfloat16 an 8-bit significand, and the colour-gradient interface is steered
by differences of populations.  The colour masses drift by at most the
stated 1e-10 of their value per step."""
import numpy as np
import pytest

import workloads as W
from oracle.ora import Oracle

from test_parity_gpu import bubble, droplet, errors, solver

pytestmark = pytest.mark.gpu

BOUNDS = {
    ("f16", "droplet"): {"rho": 5e-6, "phi": 1e-3, "u": 3e-3, "psi": 3e-4, "C": 1e-4},
    ("f16", "bubble"): {"rho": 5e-4, "phi": 1.5e-3, "u": 1e-2, "psi": 2e-3, "C": 6e-4},
    ("bf16", "droplet"): {"rho": 3e-5, "phi": 1e-2, "u": 5e-2, "psi": 5e-3, "C": 2e-4},
    ("bf16", "bubble"): {"rho": 1e-2, "phi": 2e-2, "u": 7e-2, "psi": 7e-3, "C": 8e-3},
}


@pytest.fixture(scope="module")
def oracle_runs():
    out = {}
    for name, make in (("droplet", droplet), ("bubble", bubble)):
        cfg = make()
        f = W.initial_fields(cfg, seed=7, noise=0.02)
        o = Oracle(cfg)
        o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
        o.step(1000)
        out[name] = (cfg, f, o.fields())
    return out


@pytest.mark.parametrize("storage,case", [("f16", "droplet"), ("f16", "bubble"),
                                          ("bf16", "droplet"), ("bf16", "bubble")])
def test_shifted_16bit_storage(oracle_runs, storage, case):
    cfg, f, ref = oracle_runs[case]
    s = solver(cfg, storage)
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    d0 = s.diagnostics()
    s.step(1000)
    got = s.fields()
    d = s.diagnostics()
    err = errors(ref, got)
    print(storage, case, {k: "%.1e" % v for k, v in err.items()})
    for k in got:
        assert np.isfinite(got[k]).all()
    bound = BOUNDS.get((storage, case))
    if bound:
        for k, b in bound.items():
            assert err[k] <= b, (k, err[k], b)
        for k in ("mass_R", "mass_B"):
            assert abs(d[k] - d0[k]) / d0[k] / 1000 <= 1e-10, (k, d[k], d0[k])
    s.close()
