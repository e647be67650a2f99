"""Step-level pins of the oracle's surfactant update for t >= 1 (Sec. 2.2,
Eqs. 23-24 with Eq. 28), of its moving-wall bounce-back and of its
diagnostics (Eqs. 33-34, Sec. 3.4), each against an independent
computation in the test:

  - the Adams-Bashforth / Crank-Nicolson recurrence of Eqs. 23-24 on a flat
    interface at rest, predicted step by step with the test's own sparse
    assembly of Eq. 28 and a direct solve (catches swapped or missing AB2
    coefficients, a stale or missing history S^{t-1}, weights of the wrong
    time level and a wrong diffusion half on either side);
  - the advection term of Eqs. 25-27 inside a whole step: a bulk-surfactant
    bump in a uniform flow moves downstream at the flow speed (catches a
    sign error, a missing weight in the flux, the wrong upwind side);
  - the Crank-Nicolson amplification of a Fourier mode inside a whole step;
  - Couette flow between a resting and a moving wall (2D, and D3Q19 with
    both walls moving): the half-way bounce-back with the wall term of
    reading R22 gives the exact linear profile (catches a flipped sign, a
    wrong factor or the wrong wall);
  - the diagnostics of a hand-built state whose mean velocity, centroid,
    second moments, radius, interface psi statistics and masses are known
    in closed form."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle.ora import Oracle


def lap_matrix(w, wall):
    """L_w of Eq. 28 on a [z][y][x] grid: sum over faces of the face weight
    (w_c + w_nb)/2 times (x_nb - x_c); no flux through a walled face.
    Written here from the equation, independently of the oracle."""
    nz, ny, nx = w.shape
    N = w.size
    wf = w.ravel()
    rows, cols, vals = [], [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = (z * ny + y) * nx + x
                for ax, n in ((0, nx), (1, ny), (2, nz)):
                    if n == 1:
                        continue
                    for d in (-1, 1):
                        p = [x, y, z]
                        p[ax] += d
                        if not 0 <= p[ax] < n:
                            if wall[ax]:
                                continue
                            p[ax] %= n
                        j = (p[2] * ny + p[1]) * nx + p[0]
                        f = 0.5 * (wf[c] + wf[j])
                        rows += [c, c]
                        cols += [j, c]
                        vals += [f, -f]
    return sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()


def flat_interface(nx=6, ny=32, Ds=0.08, Db=0.05):
    """Red slab |y - cy| < 8 across a periodic box, equal densities, no
    surface tension and no gravity: nothing drives a flow, the total
    populations stay at rest and the surfactant equations reduce to
    reaction + diffusion with the interface weights of the current colour
    profile (which still relaxes towards the recolouring's own profile)."""
    c = W.base(nx, ny)
    c.update(sigma0=0.0, E0=0.0, source=0, ra=0.05, rd=0.02, psi_inf=1.0, Ds=Ds, Db=Db,
             R=8.0, C0=0.5, psi0=0.3, sor_tol=1e-14)
    return c


def slab_fields(cfg, seed=3):
    nz, ny, nx = 1, cfg["ny"], cfg["nx"]
    y = np.arange(ny, dtype=np.float64)[None, :, None] * np.ones((nz, ny, nx))
    phi = np.tanh((cfg["R"] - np.abs(y - (ny - 1) / 2.0)) / cfg["width"])
    rng = np.random.default_rng(seed)
    psi = cfg["psi0"] * (1.0 - phi ** 2) * (1.0 + 0.1 * rng.uniform(-1, 1, phi.shape))
    C = cfg["C0"] * 0.5 * (1.0 - phi) * (1.0 + 0.1 * rng.uniform(-1, 1, phi.shape))
    return phi, psi, C


@pytest.mark.parametrize("Ds,Db", [(0.0, 0.0), (0.08, 0.05)], ids=["reaction", "reaction_diffusion"])
def test_ab2_crank_nicolson_recurrence(Ds, Db):
    """Eqs. 23-24: (W^{t+1} - h L^{t+1}) x^{t+1} = W^t x^t + h L^t x^t + E^t,
    E^0 = S^0 (Euler), E^t = 3/2 S^t - 1/2 S^{t-1} (AB2), with
    W = |grad rhoN| + eps_w (psi) or 1 - rhoN + eps_w (C), h = D/2,
    S = |grad rhoN| j, B = -|grad rhoN| j, j = r_a C (psi_inf - psi) - r_d psi
    (Eq. 22; u = 0), then one common rescale factor (reading R14).  Six
    steps predicted from the oracle's colour weights of each time level."""
    cfg = flat_interface(Ds=Ds, Db=Db)
    phi, psi, C = slab_fields(cfg)
    o = Oracle(cfg)
    o.init_fields(phi, psi, C)
    eps = cfg["eps_w"]
    ra, rd, pinf = cfg["ra"], cfg["rd"], cfg["psi_inf"]
    wall = cfg["wall"]
    m = o.macro()
    f = o.fields()
    a_n, rN_n, psi_n, C_n = m["a"], m["rhoN"], f["psi"], f["C"]
    assert np.abs(m["u"]).max() < 1e-14  # nothing drives a flow
    M0 = ((a_n + eps) * psi_n + (1 - rN_n + eps) * C_n).sum()
    Sp = Bp = None
    for n in range(6):
        j = ra * C_n * (pinf - psi_n) - rd * psi_n
        S, B = a_n * j, -a_n * j
        ES = S if n == 0 else 1.5 * S - 0.5 * Sp
        EB = B if n == 0 else 1.5 * B - 0.5 * Bp
        o.step(1)
        m1 = o.macro()
        a1, rN1 = m1["a"], m1["rhoN"]
        pred = []
        for x_n, w_n, w_1, h, E in ((psi_n, a_n + eps, a1 + eps, 0.5 * Ds, ES),
                                    (C_n, 1 - rN_n + eps, 1 - rN1 + eps, 0.5 * Db, EB)):
            rhs = w_n.ravel() * x_n.ravel() + h * (lap_matrix(w_n, wall) @ x_n.ravel()) + E.ravel()
            A = sp.diags(w_1.ravel()) - h * lap_matrix(w_1, wall)
            pred.append(spla.spsolve(A.tocsc(), rhs).reshape(x_n.shape))
        s = M0 / ((a1 + eps) * pred[0] + (1 - rN1 + eps) * pred[1]).sum()
        got = o.fields()
        for name, p in zip(("psi", "C"), pred):
            ref = s * p
            err = np.abs(got[name] - ref).max() / np.abs(ref).max()
            assert err < 1e-11, (n, name, err)
        a_n, rN_n, psi_n, C_n = a1, rN1, got["psi"], got["C"]
        Sp, Bp = S, B


def single_phase(nx, ny, nz=1, **kw):
    """All blue (rho^N = -1, so 1 - rho^N = 2 and |grad rho^N| = 0), no
    surface tension: a uniform flow stays uniform."""
    c = W.base(nx, ny, nz)
    c.update(sigma0=0.0, E0=0.0, R=-1e3, C0=0.0, psi0=0.0, sor_tol=1e-14)
    c.update(kw)
    return c


def test_weno_advection_moves_bulk_surfactant_downstream():
    """Eqs. 21, 24-27 in a uniform flow U along +x: (chi+eps) dC/dt =
    -d(C chi U)/dx with chi = 2, so a smooth bump of C moves at 2U/(2+eps)
    = U (1 - 5e-7).  The centroid after 80 steps (4 cells) matches to 0.5 %,
    and the bump keeps its total; flipping U moves it the other way."""
    for sign in (1.0, -1.0):
        U = 0.05 * sign
        cfg = single_phase(64, 4, Ds=0.0, Db=0.0, transport=1)
        nz, ny, nx = 1, 4, 64
        x = np.arange(nx, dtype=np.float64)[None, None, :] * np.ones((nz, ny, nx))
        x0 = 30.0
        C = 0.4 * np.exp(-((x - x0) ** 2) / (2 * 4.0 ** 2))
        u = np.zeros((3, nz, ny, nx))
        u[0] = U
        o = Oracle(cfg)
        o.init_fields(-np.ones((nz, ny, nx)), np.zeros((nz, ny, nx)), C, u)
        steps = 80
        o.step(steps)
        f = o.fields()
        assert np.abs(f["u"][0] - U).max() < 1e-15
        c1 = f["C"]
        xc = (x * c1).sum() / c1.sum()
        moved = xc - x0
        assert moved == pytest.approx(U * steps, rel=5e-3), moved
        assert c1.sum() == pytest.approx(C.sum(), rel=1e-12)


def test_crank_nicolson_mode_decay_inside_the_step():
    """Eqs. 23-24 with constant weights (one phase at rest, u = 0, no
    source): every step multiplies a Fourier mode of psi (weight eps_w) and
    of C (weight 2 + eps_w) by (1 - h lam)/(1 + h lam), h = D/2,
    lam = 2 - 2 cos k; the means stay.  Five steps of the whole update."""
    nx, ny = 32, 4
    cfg = single_phase(nx, ny, Ds=0.3, Db=0.1, transport=1)
    x = np.arange(nx, dtype=np.float64)[None, None, :] * np.ones((1, ny, nx))
    kp, kc = 2 * np.pi * 3 / nx, 2 * np.pi / nx
    psi = 0.2 + 0.05 * np.cos(kp * x)
    C = 0.5 + 0.1 * np.cos(kc * x + 0.3)
    o = Oracle(cfg)
    o.init_fields(-np.ones_like(x), psi, C)
    n = 5
    o.step(n)
    f = o.fields()
    Gp = (1 - 0.5 * cfg["Ds"] * (2 - 2 * np.cos(kp))) / (1 + 0.5 * cfg["Ds"] * (2 - 2 * np.cos(kp)))
    Gc = (1 - 0.5 * cfg["Db"] * (2 - 2 * np.cos(kc))) / (1 + 0.5 * cfg["Db"] * (2 - 2 * np.cos(kc)))
    assert np.allclose(f["psi"], 0.2 + 0.05 * Gp ** n * np.cos(kp * x), rtol=0, atol=1e-12)
    assert np.allclose(f["C"], 0.5 + 0.1 * Gc ** n * np.cos(kc * x + 0.3), rtol=0, atol=1e-12)


def couette(D):
    """Walls half-way beyond the ends of the wall axis (y in 2D, z in 3D);
    2D: low wall at rest, high wall moving +U along x; 3D: walls moving -U
    and +U along x (the Sec. 3.3 shear set-up)."""
    U = 2e-4
    if D == 2:
        c = single_phase(4, 12, muB0=0.3, muR0=0.3, transport=0)
        c["wall"] = [0, 1, 0]
        c["uw_hi"] = [[0.0] * 3, [U, 0.0, 0.0], [0.0] * 3]
        lo, hi, n = 0.0, U, 12
    else:
        c = single_phase(4, 4, 10, muB0=0.3, muR0=0.3, transport=0)
        c["wall"] = [0, 0, 1]
        c["uw_lo"] = [[0.0] * 3, [0.0] * 3, [-U, 0.0, 0.0]]
        c["uw_hi"] = [[0.0] * 3, [0.0] * 3, [U, 0.0, 0.0]]
        lo, hi, n = -U, U, 10
    return c, lo, hi, n


@pytest.mark.parametrize("D", [2, 3])
def test_couette_profile_between_moving_walls(D):
    """Reading R22 (moving-wall bounce-back, f_i = f_opp + 2 w_i rho (e_i . u_w)
    / c_s^2 per colour) and the half-way wall position: the steady flow
    between walls at -1/2 and n - 1/2 is linear,
    u_x = u_lo + (u_hi - u_lo)(k + 1/2)/n, with no velocity across.  The
    lattice's compressibility bends the profile at second order in the wall
    speed (relative deviation ~1e-2 U: 4e-6 at U = 0.02); at U = 2e-4 the
    profile is linear to 2e-9 of the wall speed."""
    cfg, lo, hi, n = couette(D)
    o = Oracle(cfg)
    shape = o.shape
    o.init_fields(-np.ones(shape), np.zeros(shape), np.zeros(shape))
    o.step(3000)
    u = o.fields()["u"]
    k = np.arange(n) + 0.5
    exact = lo + (hi - lo) * k / n
    prof = u[0].mean(axis=(0, 2)) if D == 2 else u[0].mean(axis=(1, 2))
    assert np.abs(prof - exact).max() < 2e-9 * abs(hi - lo), prof - exact
    full = exact[None, :, None] if D == 2 else exact[:, None, None]
    assert np.abs(u[0] - full).max() < 2e-9 * abs(hi - lo)
    assert np.abs(u[1:]).max() < 1e-10 * abs(hi - lo)


def hand_built(D):
    """A state with sharp, known regions: a red box (rho^N = 1), a few blue
    interface cells with rho^N = -0.3 (psi statistics over |rho^N| < 0.5),
    blue elsewhere; a prescribed velocity field; no surface tension or
    gravity, so the force vanishes and u is the prescribed field."""
    if D == 2:
        shape, box = (1, 30, 40), (slice(0, 1), slice(5, 21), slice(10, 20))
    else:
        shape, box = (14, 12, 10), (slice(3, 11), slice(2, 8), slice(4, 9))
    nz, ny, nx = shape
    c = W.base(nx, ny, nz)
    c.update(sigma0=0.0, E0=0.0, rhoR0=1.0, rhoB0=1.0, transport=0, muB0=0.2)
    phi = -np.ones(shape)
    phi[box] = 1.0
    iface = [(0, 2, 3), (0, 25, 30), (0, 27, 1)] if D == 2 else [(1, 1, 1), (12, 10, 0), (0, 5, 7)]
    psi = np.zeros(shape)
    vals = [0.3, 0.7, 0.45]
    for p, v in zip(iface, vals):
        phi[p] = -0.3
        psi[p] = v
    z, y, x = np.meshgrid(*(np.arange(s, dtype=np.float64) for s in shape), indexing="ij")
    u = np.zeros((3,) + shape)
    u[0] = 0.01 + 1e-4 * x - 2e-4 * y
    u[1] = -0.02 + 3e-4 * y + 1e-4 * (x % 3)
    if D == 3:
        u[2] = 0.005 - 2e-4 * z + 1e-4 * x
    return c, phi, psi, u, box, vals, (x, y, z)


@pytest.mark.parametrize("D", [2, 3])
def test_diagnostics_of_a_hand_built_state(D):
    """Eqs. 33-34 and Sec. 3.4: U is the mean velocity over rho^N >= 0, the
    centroid and second moments those of that region (a box of w x h (x d)
    cells: sum (x - cx)^2 = h w (w^2 - 1)/12 per axis), AR = sqrt(I_hor /
    I_vert) with the vertical axis the last one when g = 0, R from the area
    (2D: sqrt(n / pi)) or volume (3D: cbrt(3 n / (4 pi))), Re = 2 rhoB0
    |U_vert| R / muB0; psi statistics over |rho^N| < 0.5; colour masses
    rho^k0 (1 +- rho^N)/2 summed; umax the largest |u|."""
    cfg, phi, psi, u, box, vals, (x, y, z) = hand_built(D)
    o = Oracle(cfg)
    o.init_fields(phi, psi, np.zeros_like(phi), u)
    d = o.diagnostics()
    red = phi >= 0
    n = red.sum()
    U = [u[a][red].mean() for a in range(3)]
    for a in range(D):
        assert d["U"][a] == pytest.approx(U[a], rel=1e-12, abs=1e-15)
    cen = [x[red].mean(), y[red].mean(), z[red].mean()]
    for a in range(D):
        assert d["centroid"][a] == pytest.approx(cen[a], rel=1e-13)
    sides = [box[2].stop - box[2].start, box[1].stop - box[1].start, box[0].stop - box[0].start]
    vol = int(np.prod(sides[:D]))

    def second(a):
        return vol // sides[a] * sides[a] * (sides[a] ** 2 - 1) / 12.0

    vert, hor = D - 1, 0
    assert d["aspect_ratio"] == pytest.approx(math.sqrt(second(hor) / second(vert)), rel=1e-12)
    R = math.sqrt(n / math.pi) if D == 2 else (3 * n / (4 * math.pi)) ** (1 / 3)
    assert d["Re"] == pytest.approx(2 * cfg["rhoB0"] * abs(U[vert]) * R / cfg["muB0"], rel=1e-12)
    assert d["psi_av"] == pytest.approx(np.mean(vals), rel=1e-13)
    assert d["psi_min"] == min(vals) and d["psi_max"] == max(vals)
    assert d["umax"] == pytest.approx(np.sqrt((u ** 2).sum(axis=0)).max(), rel=1e-13)
    assert d["mass_R"] == pytest.approx((cfg["rhoR0"] * 0.5 * (1 + phi)).sum(), rel=1e-14)
    assert d["mass_B"] == pytest.approx((cfg["rhoB0"] * 0.5 * (1 - phi)).sum(), rel=1e-14)
