"""Pins of the mirror (symmetry) planes of Sec. 3.1 in the oracle (no GPU).

A grid with mirror planes half-way beyond both ends of an axis is the
restriction of a periodic grid twice as long whose fields are mirror-
symmetric about those planes: a droplet centred at the junction of four (2D)
or eight (3D) quarter / octant domains.  Run on both grids, the quarter or
octant must equal the restriction of the full run to rounding.  This pins
the specular reflection of the populations, the free-slip ghost velocity of
the correction and FD stencils, the mirrored scalars and the zero flux of
the surfactant faces together: a wrong direction, sign or index in any of
them breaks the equality.  A uniform flow along a mirror plane is an exact
steady state (free slip); along a bounce-back wall it is not."""
import numpy as np
import pytest

import workloads as W
from oracle.ora import Oracle


def _sym_fields(cfg, full_n, U=1e-3):
    """Fields of a droplet centred at (n - 1/2) on a periodic grid of 2n
    cells per axis, with a velocity odd about the mirror planes of its normal
    component and even about the others."""
    f = W.initial_fields(cfg)
    D = 2 if cfg.get("nz", 1) == 1 else 3
    shape = f["phi"].shape  # (nz, ny, nx)
    u = np.zeros((3,) + shape)
    half = [full_n[a] // 2 for a in range(3)]
    coords = np.meshgrid(*[np.arange(shape[2 - a]) for a in (2, 1, 0)], indexing="ij")
    z, y, x = coords
    X = [x, y, z]
    s = [np.pi * (X[a] - (half[a] - 0.5)) / max(half[a], 1) for a in range(3)]
    for a in range(D):
        v = U * np.sin(s[a])
        for b in range(D):
            if b != a:
                v = v * np.cos(s[b])
        u[a] = v
    f["u"] = u
    return f


def _run_pair(full_cfg, part_cfg, steps):
    n = [full_cfg["nx"], full_cfg["ny"], full_cfg.get("nz", 1)]
    f = _sym_fields(full_cfg, n)
    D = 2 if n[2] == 1 else 3
    sl = (slice(n[2] // 2, None) if D == 3 else slice(None), slice(n[1] // 2, None),
          slice(n[0] // 2, None))
    full = Oracle(full_cfg)
    full.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    part = Oracle(part_cfg)
    part.init_fields(f["phi"][sl], f["psi"][sl], f["C"][sl],
                     np.ascontiguousarray(f["u"][(slice(None),) + sl]))
    d0 = part.diagnostics()
    full.step(steps)
    part.step(steps)
    a, b = full.fields(), part.fields()
    for k in ("rho", "phi", "psi", "C"):
        ref = a[k][sl]
        err = np.abs(b[k] - ref).max() / np.abs(ref).max()
        assert err <= 1e-11, (k, err)
    ref = a["u"][(slice(None),) + sl]
    err = np.abs(b["u"] - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, ("u", err)
    d = part.diagnostics()
    for k in ("mass_R", "mass_B", "surf_total"):
        assert abs(d[k] - d0[k]) <= 1e-12 * d0[k], k
    return b


def test_quarter_with_mirror_planes_equals_full_grid_2d():
    full = W.droplet_adsorption_2d(n=40, R=8.0, C0=0.5)
    full.update(ny=32, center=[19.5, 15.5, 0.0], psi0=0.3)
    part = dict(full, nx=20, ny=16, wall=[2, 2, 0], center=[-0.5, -0.5, 0.0])
    b = _run_pair(full, part, 30)
    assert np.abs(b["u"]).max() > 1e-4  # the flow is not trivial


def test_quarter_density_ratio_10_2d():
    """The same with a light droplet (density ratio 10, no gravity): the
    heavy phase's alpha makes the correction term of Eq. 37 act, and with it
    the ghost velocity of its stencil at the mirror planes."""
    full = W.bubble_rise_2d(nx=36, ny=32, D_b=14.0)
    full.update(g=[0.0, 0.0, 0.0], center=[17.5, 15.5, 0.0], sigma0=0.01, psi0=0.5,
                wall=[0, 0, 0])
    part = dict(full, nx=18, ny=16, wall=[2, 2, 0], center=[-0.5, -0.5, 0.0])
    _run_pair(full, part, 30)


@pytest.mark.parametrize("ratio", [1, 10])
def test_octant_with_mirror_planes_equals_full_grid_3d(ratio):
    full = W.droplet_adsorption_2d(n=20, R=4.5, C0=0.5)
    aR, aB = W._alphas(3, 1.0 / ratio, 1.0)
    full.update(ny=16, nz=18, alphaR=aR, alphaB=aB, rhoR0=1.0 / ratio,
                center=[9.5, 7.5, 8.5], psi0=0.3)
    part = dict(full, nx=10, ny=8, nz=9, wall=[2, 2, 2], center=[-0.5, -0.5, -0.5])
    _run_pair(full, part, 12)


@pytest.mark.parametrize("nz", [1, 6])
def test_uniform_flow_along_mirror_planes_is_steady(nz):
    """Free slip: a uniform single-phase flow parallel to mirror planes is
    unchanged by the step (the mirror image of its equilibrium populations is
    itself); between bounce-back walls the same flow is slowed at the walls."""
    n = 10
    out = {}
    for wall in (2, 1):
        c = W.base(n, 8, nz)
        a = W._alphas(2 if nz == 1 else 3, 1.0, 1.0)
        c.update(rhoR0=1.0, rhoB0=1.0, alphaR=a[0], alphaB=a[1], muR0=0.1, muB0=0.1,
                 transport=0, sigma0=0.0, wall=[wall, 0, 0])
        phi = -np.ones((nz, 8, n))
        u = np.zeros((3, nz, 8, n))
        u[1] = 0.02
        o = Oracle(c)
        o.init_fields(phi, np.zeros_like(phi), np.zeros_like(phi), u)
        o.step(50)
        out[wall] = o.fields()["u"]
    assert np.abs(out[2][1] - 0.02).max() <= 1e-13
    assert np.abs(out[2][0]).max() <= 1e-15 and np.abs(out[2][2]).max() <= 1e-15
    assert out[1][1][..., 0].max() < 0.019  # no slip at the walls
