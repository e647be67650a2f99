"""The droplet migration test of Sec. 3.2 in 3D (insoluble surfactant held
at psi = psi_inf z / L_z, linear equation of state, walls on x and y,
periodic z) on the GPU.

  - Parity: a small box (R = 4) against the oracle in FP64.
  - Physics: the steady droplet velocity U of Eqs. 33-34 against the YGB
    velocity of Eq. 32.  The paper prints U/U_YGB = 0.958 in the 5R x 5R x
    10R box and 0.993 in the 10R cube at R = 30; at the resolutions a test
    affords (FP32, measured): 1.025 (5R x 5R x 10R, R = 10), 1.084 (10R
    cube, R = 10), 0.984 (5R x 5R x 10R, R = 15).  The test checks the ratio
    within 10 % of 1, the slowing by the walls of the narrower box (0.946 at
    R = 10; 0.965 in the paper), and the approach to the printed 0.958 as R
    grows."""
import numpy as np
import pytest

import workloads as W
from oracle.ora import Oracle

from test_parity_gpu import errors, solver

pytestmark = pytest.mark.gpu


def test_small_migration_matches_oracle():
    cfg = W.migration_3d(R=4)
    f = W.initial_fields(cfg, seed=9, u0=1e-4)
    o = Oracle(cfg)
    o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    s = solver(cfg, "f64")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    o.step(30)
    s.step(30)
    err = errors(o.fields(), s.fields())
    s.close()
    assert max(err.values()) < 1e-9, err


def _terminal(R, shape, steps):
    """U/U_YGB averaged over the last quarter of `steps` (sampled every 500
    steps; the velocity is steady after about 8 R^2 / nu steps)."""
    cfg = W.migration_3d(R, shape)
    f = W.initial_fields(cfg)
    s = solver(cfg, "f32")
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    ygb = W.migration_ygb(cfg)
    u, done = [], 0
    for t in range(500, steps + 1, 500):
        s.step(t - done)
        done = t
        u.append(s.diagnostics()["U"][2] / ygb)
    s.close()
    return float(np.mean(u[-len(u) // 4:]))


@pytest.fixture(scope="module")
def terminal():
    return {"box10": _terminal(10, (5, 5, 10), 16000),
            "cube10": _terminal(10, (10, 10, 10), 24000),
            "box15": _terminal(15, (5, 5, 10), 20000)}


def test_terminal_velocity_against_ygb(terminal):
    for k, v in terminal.items():
        assert 0.9 <= v <= 1.1, (k, v)


def test_wall_confinement_and_resolution(terminal, printed):
    ratio = terminal["box10"] / terminal["cube10"]
    assert 0.90 <= ratio <= 0.99, ratio
    box = printed["migration_5Rx5Rx10R"]
    assert abs(terminal["box15"] - box) < abs(terminal["box10"] - box), terminal
