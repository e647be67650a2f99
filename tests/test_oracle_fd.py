"""Pins of the oracle's finite-difference operators (Sec. 2.1 isotropic
gradient, Sec. 2.2 WENO3, diffusion operator of Eq. 28, SOR) against
polynomial exactness, convergence order, closed-form Fourier symbols,
conservation / symmetry invariants and a direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads
from oracle.ora import Oracle


def ctx(nx, ny, nz=1, wall=(0, 0, 0)):
    c = workloads.base(nx, ny, nz)
    c["wall"] = list(wall)
    return Oracle(c)


def grid(o):
    nz, ny, nx = o.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(float), y.astype(float), z.astype(float)


@pytest.mark.parametrize("nz", [1, 8])
def test_isotropic_gradient_exact_on_quadratics(nz):
    """Sec. 2.1 (after Eq. 9): the isotropic stencil sum_i w_i X(x+e_i) e_i / c_s^2
    reproduces the gradient of any quadratic exactly (second-order lattice
    isotropy); checked away from the periodic seam."""
    o = ctx(10, 9, nz)
    x, y, z = grid(o)
    X = 0.3 * x * x - 0.2 * x * y + 0.1 * y * y + 0.7 * x - 0.4 * y + 2.0
    ex = [0.6 * x - 0.2 * y + 0.7, -0.2 * x + 0.2 * y - 0.4, 0 * x]
    if nz > 1:
        X = X + 0.05 * z * z + 0.3 * x * z - 0.1 * z
        ex[0] = ex[0] + 0.3 * z
        ex[2] = 0.1 * z + 0.3 * x - 0.1
    G = o.iso_grad(X)
    s = (slice(1, -1) if nz > 1 else slice(None), slice(1, -1), slice(1, -1))
    for a in range(3 if nz > 1 else 2):
        assert np.allclose(G[a][s], ex[a][s], atol=1e-12)


def test_isotropic_gradient_mirror_at_walls():
    """Reading R21: scalars are mirrored about a half-way wall, so a field
    symmetric about the channel centre has zero normal gradient there and an
    antisymmetric gradient."""
    o = ctx(12, 8, wall=(1, 0, 0))
    x, y, _ = grid(o)
    X = np.cos(np.pi * (x + 0.5) / 12) ** 2 + 0.1 * np.sin(2 * np.pi * y / 8)
    G = o.iso_grad(X)
    assert np.allclose(G[0], -G[0][:, :, ::-1], atol=1e-14)
    assert np.allclose(G[1], G[1][:, :, ::-1], atol=1e-14)


def test_weno_exact_on_quadratics_both_sides():
    """Eqs. 26-27: both one-sided WENO3 differences are exact for quadratic
    data whatever the nonlinear weights; the divergence of a quadratic flux
    therefore equals its exact derivative for either sign of u."""
    o = ctx(16, 14)
    x, y, _ = grid(o)
    Psi = np.stack([0.2 * x * x - x + 3, 0.1 * y * y + 0.3 * y - 1, 0 * x])
    exact = 0.4 * x - 1 + 0.2 * y + 0.3
    s = (slice(None), slice(2, -2), slice(2, -2))
    for sgn in (1.0, -1.0, 0.0):
        u = np.stack([sgn * np.ones_like(x), -sgn * np.ones_like(x), 0 * x])
        assert np.allclose(o.weno_div(Psi, u)[s], exact[s], atol=1e-12)


def test_weno_third_order_convergence():
    """Sec. 2.2 names a third-order WENO scheme: on smooth periodic data the
    error of div Psi falls by ~2^3 per grid doubling."""
    errs = []
    for n in (32, 64, 128):
        o = ctx(n, 1)
        x, _, _ = grid(o)
        k = 2 * np.pi / n
        Psi = np.stack([np.sin(k * x) * 1e-2, 0 * x, 0 * x])
        u = np.stack([np.ones_like(x), 0 * x, 0 * x])
        err = np.abs(o.weno_div(Psi, u) - 1e-2 * k * np.cos(k * x)).max()
        errs.append(err / (1e-2 * k))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.7), rates


def test_weno_upwind_stencil_support():
    """Eq. 25 (reading R9): for u_x > 0 only {i-2..i+1} enter, for u_x < 0 only
    {i-1..i+2}: a perturbation outside the stencil leaves div unchanged."""
    o = ctx(16, 1)
    rng = np.random.default_rng(0)
    Psi = np.zeros((3, 1, 1, 16))
    Psi[0] = rng.normal(size=(1, 1, 16))
    for sgn, far in ((1.0, 2), (-1.0, -2)):
        u = np.zeros_like(Psi)
        u[0] = sgn
        d0 = o.weno_div(Psi, u)
        P2 = Psi.copy()
        P2[0, 0, 0, 8 + far] += 1.0
        d1 = o.weno_div(P2, u)
        assert d1[0, 0, 8] == d0[0, 0, 8]


def test_diffusion_operator_invariants_and_symbol():
    """Eq. 28: flux form with face weights (w_c + w_nb)/2, so sum L_w x = 0
    (periodic and walled), L_w is symmetric and L_w 1 = 0; for constant w it
    is w times the 5-point Laplacian, whose Fourier symbol is
    -(4 - 2 cos kx - 2 cos ky)."""
    rng = np.random.default_rng(5)
    for wall in ((0, 0, 0), (1, 0, 0), (1, 1, 0)):
        o = ctx(12, 10, wall=wall)
        w = rng.uniform(0.01, 1.0, o.shape)
        x1, x2 = rng.normal(size=o.shape), rng.normal(size=o.shape)
        L1, L2 = o.diffuse(w, x1), o.diffuse(w, x2)
        assert abs(L1.sum()) < 1e-12
        assert np.isclose((x2 * L1).sum(), (x1 * L2).sum(), rtol=1e-12)
        assert np.allclose(o.diffuse(w, np.ones(o.shape)), 0, atol=1e-15)
    o = ctx(16, 12)
    x, y, _ = grid(o)
    kx, ky = 2 * np.pi * 3 / 16, 2 * np.pi * 2 / 12
    mode = np.cos(kx * x + ky * y)
    L = o.diffuse(np.full(o.shape, 0.7), mode)
    assert np.allclose(L, -0.7 * (4 - 2 * np.cos(kx) - 2 * np.cos(ky)) * mode, atol=1e-13)


def _assemble(o, w, h):
    """(W - h L_W) as a sparse matrix, from the face weights of Eq. 28."""
    nz, ny, nx = o.shape
    wall = o.cfg["wall"]
    N = nx * ny * nz
    wf = w.ravel()
    rows, cols, vals = [], [], []
    diag = wf.copy()
    for yy in range(ny):
        for xx in range(nx):
            c = yy * nx + xx
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                X, Y = xx + dx, yy + dy
                if not (0 <= X < nx):
                    if wall[0]:
                        continue
                    X %= nx
                if not (0 <= Y < ny):
                    if wall[1]:
                        continue
                    Y %= ny
                j = Y * nx + X
                f = 0.5 * (wf[c] + wf[j])
                diag[c] += h * f
                rows.append(c)
                cols.append(j)
                vals.append(-h * f)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr() + sp.diags(diag)
    return A


@pytest.mark.parametrize("wall", [(0, 0, 0), (1, 0, 0)])
def test_sor_reaches_the_direct_solution(wall):
    """Sec. 2.2: the CN systems are SPD and SOR with omega = 1.2 solves them;
    the converged iterate equals a sparse direct solve (scipy spsolve) of the
    same system, including the tiny-weight rows of the regularised weights."""
    o = ctx(14, 12, wall=wall)
    rng = np.random.default_rng(6)
    x, y, _ = grid(o)
    w = np.abs(np.tanh((6.0 - np.hypot(x - 6.5, y - 5.5)) / 2.0)) ** 4 + 1e-6
    w = w * (1 + 0.1 * rng.uniform(size=o.shape))
    rhs = rng.normal(size=o.shape) * w
    sol, it = o.sor(w, 0.05, rhs, np.zeros(o.shape))
    assert it > 0
    ref = spla.spsolve(_assemble(o, w, 0.05).tocsc(), rhs.ravel()).reshape(o.shape)
    assert np.abs(sol - ref).max() <= 1e-11 * np.abs(ref).max()


def test_crank_nicolson_fourier_amplification():
    """Eqs. 23-24 with constant weight, no convection and no source: one CN step
    multiplies a Fourier mode by (1 - D lam / 2)/(1 + D lam / 2), lam = 4 - 2cos kx
    - 2cos ky; the oracle's SOR reproduces it."""
    o = ctx(16, 16)
    x, y, _ = grid(o)
    kx, ky = 2 * np.pi / 16, 2 * np.pi * 3 / 16
    m = np.cos(kx * x) * np.cos(ky * y)
    Dd = 0.1
    w = np.ones(o.shape)
    rhs = m + 0.5 * Dd * o.diffuse(w, m)
    sol, _ = o.sor(w, 0.5 * Dd, rhs, m)
    lam = 4 - 2 * np.cos(kx) - 2 * np.cos(ky)
    assert np.allclose(sol, (1 - Dd * lam / 2) / (1 + Dd * lam / 2) * m, atol=1e-12)
