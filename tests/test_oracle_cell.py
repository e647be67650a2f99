"""Pins of the oracle's cell-level building blocks against what the paper and
the mathematics fix (no GPU).

Each test names the passage it checks.  None of them re-types the oracle's
formula: they check an independent property (a moment identity, a closed
form derived by hand, an invariant) that a transcription mistake would break.
"""
import itertools

import numpy as np
import pytest

from oracle import ora


def lat(D):
    return ora.lattice(D)


@pytest.mark.parametrize("D", [2, 3])
def test_lattice_isotropy(D):
    """D2Q9 / D3Q19 weights and velocities (Sec. 2.1: c_s^2 = 1/3): moments of
    w up to fourth order are those of an isotropic Gaussian."""
    e, w, _, _ = lat(D)
    e = e[:, :D].astype(float)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ e, 0.0, atol=1e-15)
    d = np.eye(D)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), d / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0.0, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) +
           np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-15)


def test_M2_rows_are_the_d2q9_moment_polynomials():
    """Eq. 36: the rows of M are rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx,
    p_xy, i.e. these polynomials of the velocities; the rows are orthogonal."""
    e, _, M, Minv = lat(2)
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    e2 = ex ** 2 + ey ** 2
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, ex,
            (-5 + 3 * e2) * ex, ey, (-5 + 3 * e2) * ey, ex ** 2 - ey ** 2, ex * ey]
    assert np.array_equal(M, np.array(rows))
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)), atol=0)
    assert np.allclose(M @ Minv, np.eye(9), atol=1e-14)


def test_M3_rows_are_the_d3q19_raw_moments():
    """Eq. 39: raw moments 1, e, |e|^2, 2ex^2-ey^2-ez^2, ey^2-ez^2, products,
    third-order and fourth-order products."""
    e, _, M, Minv = lat(3)
    x, y, z = (e[:, a].astype(float) for a in range(3))
    rows = [np.ones(19), x, y, z, x * x + y * y + z * z, 2 * x * x - y * y - z * z,
            y * y - z * z, x * y, x * z, y * z, x * x * y, x * y * y, x * x * z,
            x * z * z, y * y * z, y * z * z, x * x * y * y, x * x * z * z, y * y * z * z]
    assert np.array_equal(M, np.array(rows))
    assert np.allclose(M @ Minv, np.eye(19), atol=1e-13)


def test_meq_standard_alpha_is_textbook_bgk_equilibrium():
    """Eq. 37 at alpha = 4/9 (c_s^2 = 1/3, correction coefficient 0) gives the
    standard second-order D2Q9 equilibrium w_i rho (1 + 3 e.u + 9/2 (e.u)^2
    - 3/2 u^2)."""
    e, w, _, Minv = lat(2)
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = rng.uniform(0.5, 2)
        u = rng.uniform(-0.1, 0.1, 2)
        f = Minv @ ora.meq(2, rho, u, 4.0 / 9.0)
        eu = e[:, :2] @ u
        ref = w * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u @ u)
        assert np.allclose(f, ref, atol=1e-15)
    assert np.isclose(1.8 * 4 / 9 - 0.8, 0.0, atol=1e-15)
    assert np.isclose(ora.cs2(2, 4 / 9), 1 / 3, atol=1e-15)
    assert np.isclose(ora.cs2(3, 1 / 3), 1 / 3, atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_meq_moments_for_any_alpha(D):
    """App. A: for any alpha^k the equilibria carry density rho, momentum rho u,
    momentum flux rho c_s^2 delta + rho u u with (c_s^k)^2 = (3/5)(1-alpha) (2D)
    or (1/2)(1-alpha) (3D), and the third moment of the third-order Hermite
    expansion: sum f e_a e_b^2 = rho c_s^2 u_a (a != b)."""
    e, _, _, Minv = lat(D)
    E = e[:, :D].astype(float)
    rng = np.random.default_rng(2)
    for alpha in (0.2, 4 / 9, 1 / 3, 0.9444444444444444):
        rho = rng.uniform(0.1, 2)
        u = rng.uniform(-0.1, 0.1, D)
        f = Minv @ ora.meq(D, rho, np.r_[u, [0] * (3 - D)], alpha)
        c2 = ora.cs2(D, alpha)
        assert np.isclose(f.sum(), rho, atol=1e-14)
        assert np.allclose(f @ E, rho * u, atol=1e-14)
        P = np.einsum("i,ia,ib->ab", f, E, E)
        assert np.allclose(P, rho * c2 * np.eye(D) + rho * np.outer(u, u), atol=1e-14)
        for a, b in itertools.permutations(range(D), 2):
            assert np.isclose(np.sum(f * E[:, a] * E[:, b] ** 2), rho * c2 * u[a], atol=1e-14)
    assert np.isclose(ora.cs2(2, 0.2), 0.6 * 0.8)


def test_d3q19_equilibrium_at_rest_is_the_alpha_model_rest_state():
    """The rest state of the alpha-model on D3Q19, for any alpha^k: the rest
    particle carries rho alpha, and the moving directions share rho (1 -
    alpha) in the proportion of the standard weights, 1/18 : 1/36 over their
    total 2/3, i.e. rho (1 - alpha)/12 on the axes and rho (1 - alpha)/24 on
    the diagonals.  It pins every row of Eq. 40 at u = 0, rows 17-19 included
    (their rest value rho (1 - alpha)/6; rho/9 at the standard alpha 1/3,
    the fourth moment sum w_i e_a^2 e_b^2 of the standard lattice); only
    their velocity terms stay unpinned."""
    e, w, _, Minv = lat(3)
    axis = np.abs(e).sum(axis=1) == 1
    diag = np.abs(e).sum(axis=1) == 2
    rng = np.random.default_rng(4)
    for alpha in (0.2, 1 / 3, 0.6, 0.9444444444444444):
        rho = rng.uniform(0.1, 2)
        f = Minv @ ora.meq(3, rho, np.zeros(3), alpha)
        ref = np.where(axis, rho * (1 - alpha) / 12, np.where(diag, rho * (1 - alpha) / 24,
                                                              rho * alpha))
        assert np.allclose(f, ref, atol=1e-15), alpha
    # the standard alpha gives the standard weights
    f = Minv @ ora.meq(3, 1.0, np.zeros(3), 1 / 3)
    assert np.allclose(f, w, atol=1e-15)
    assert np.isclose(np.sum(w * e[:, 0] ** 2 * e[:, 1] ** 2), 1 / 9)


def test_correction_coefficient_is_the_lattice_third_moment_deficit():
    """App. A: 1.8 alpha - 0.8 = 1 - 3 (c_s^k)^2 (D2Q9 has sum f e_x^3 =
    sum f e_x, so the equilibrium third moment misses 3 c_s^2 - 1)."""
    for alpha in np.linspace(0.1, 0.99, 7):
        assert np.isclose(1.8 * alpha - 0.8, 1 - 3 * ora.cs2(2, alpha), atol=1e-14)
    c = ora.corr(2, [0.3, -0.1, 0])
    assert np.allclose(c, [0, 3 * 0.2, 0, 0, 0, 0, 0, 0.4, 0], atol=1e-15)
    c3 = ora.corr(3, [0.3, -0.1, 0.2])
    exp = np.zeros(19)
    exp[4], exp[5], exp[6] = 0.4, 0.6 + 0.1 - 0.2, -0.3
    assert np.allclose(c3, exp, atol=1e-15)


def test_forcing_moments_closed_form_d2q9():
    """Eq. 4 for D2Q9: the moments of the forcing term, derived by hand from
    the lattice isotropy, are (0, 6u.F, -6u.F, Fx, -Fx, Fy, -Fy,
    2(uxFx - uyFy), uxFy + uyFx)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        u, F = rng.normal(size=2) * 0.1, rng.normal(size=2) * 1e-3
        uF = u @ F
        exp = [0, 6 * uF, -6 * uF, F[0], -F[0], F[1], -F[1],
               2 * (u[0] * F[0] - u[1] * F[1]), u[0] * F[1] + u[1] * F[0]]
        assert np.allclose(ora.forcing(2, np.r_[u, 0], np.r_[F, 0]), exp, atol=1e-16)


def _cfg(**kw):
    import workloads
    c = workloads.base(8, 8)
    c.update(kw)
    return c


@pytest.mark.parametrize("D", [2, 3])
def test_collision_conserves_mass_and_adds_force(D):
    """Eqs. 1-4 and 10: the collision conserves each colour's mass after
    recolouring and changes the total momentum by exactly F, where the
    velocity fed to the collision is (sum f e + F/2)/rho (Guo forcing)."""
    e, _, _, Minv = lat(D)
    E = e[:, :D].astype(float)
    rng = np.random.default_rng(4)
    cfg = _cfg(rhoR0=0.1, rhoB0=1.0, alphaR=0.3, alphaB=0.9, muR0=0.02, muB0=0.2)
    for _ in range(5):
        rR, rB = rng.uniform(0.01, 0.1), rng.uniform(0.1, 1.0)
        u0 = rng.uniform(-0.05, 0.05, 3)
        u0[D:] = 0
        fR = Minv @ ora.meq(D, rR, u0, cfg["alphaR"]) + rng.normal(size=len(E)) * 1e-4
        fB = Minv @ ora.meq(D, rB, u0, cfg["alphaB"]) + rng.normal(size=len(E)) * 1e-4
        F = np.r_[rng.normal(size=D) * 1e-3, [0] * (3 - D)]
        rho = fR.sum() + fB.sum()
        j = (fR + fB) @ E
        u = np.r_[(j + 0.5 * F[:D]) / rho, [0] * (3 - D)]
        dR, dB = rng.normal(size=3) * 1e-3, rng.normal(size=3) * 1e-3
        g = rng.normal(size=3)
        g[D:] = 0
        fR2, fB2 = ora.collide_cell(cfg, D, fR, fB, u, F, dR, dB, g)
        assert np.isclose(fR2.sum(), fR.sum(), rtol=1e-13)
        assert np.isclose(fB2.sum(), fB.sum(), rtol=1e-13)
        assert np.allclose((fR2 + fB2) @ E, j + F[:D], atol=1e-15)


def test_recolouring_moves_red_up_the_colour_gradient():
    """Eqs. 11-12: recolouring splits f^dagger in proportion rho^k/rho plus a
    segregation term beta w_i rho^R rho^B / rho cos(theta_i)|e_i| that pushes
    red along grad rho^N and blue against it, leaving the total unchanged."""
    D = 2
    e, _, _, Minv = lat(D)
    E = e[:, :2].astype(float)
    cfg = _cfg()
    fR = Minv @ ora.meq(2, 0.5, [0, 0, 0], 4 / 9)
    fB = Minv @ ora.meq(2, 0.5, [0, 0, 0], 4 / 9)
    z = np.zeros(3)
    g = np.array([0.3, 0.0, 0.0])
    fR2, fB2 = ora.collide_cell(cfg, D, fR, fB, z, z, z, z, g)
    jR = fR2 @ E
    # red momentum along +x: beta * sum_i w_i (rR rB/rho) e_ix (e_ix gx)/|g| = beta rR rB/rho / 3
    assert np.isclose(jR[0], 0.7 * 0.25 / 3.0, rtol=1e-10)
    assert np.isclose(jR[1], 0.0, atol=1e-16)
    assert np.allclose((fR2 + fB2) @ E, 0.0, atol=1e-16)


def test_eos_langmuir_closed_forms():
    """Eq. 8 and Sec. 2.1: sigma(0) = sigma0; sigma reaches sigma_min =
    sigma0/10 at CMC = psi_inf (1 - exp(-0.9/E0)) and stays there; the
    Marangoni coefficient of Eq. 9 is -d sigma / d psi = sigma0 E0/(psi_inf - psi)
    below the CMC and 0 above it."""
    cfg = _cfg(sigma0=0.1, E0=0.5, psi_inf=2.0)
    cmc = ora.cmc(cfg)
    assert np.isclose(cmc, 2.0 * (1 - np.exp(-0.9 / 0.5)), rtol=1e-15)
    s0, m0 = ora.eos(cfg, 0.0)
    assert np.isclose(s0, 0.1) and np.isclose(m0, 0.1 * 0.5 / 2.0)
    s_below, _ = ora.eos(cfg, cmc * (1 - 1e-9))
    assert np.isclose(s_below, 0.01, rtol=1e-7)
    for psi in (cmc, cmc * 1.1, 5.0):
        s, m = ora.eos(cfg, psi)
        assert s == pytest.approx(0.01) and m == 0.0
    for psi in (0.1, 0.5, 1.0):
        h = 1e-6
        ds = (ora.eos(cfg, psi + h)[0] - ora.eos(cfg, psi - h)[0]) / (2 * h)
        assert np.isclose(-ds, ora.eos(cfg, psi)[1], rtol=1e-7)
    clean = _cfg(sigma0=0.1, E0=0.0, psi_inf=1.0)
    for psi in (0.0, 0.5, 3.0):  # E0 = 0: constant tension, no Marangoni stress
        assert ora.eos(clean, psi) == (0.1, 0.0)
    lin = _cfg(sigma0=0.001, E0=0.5, psi_inf=1.0, eos=1)
    assert ora.eos(lin, 0.4) == pytest.approx((0.001 * 0.8, 0.001 * 0.5))


def test_recolouring_weight_is_the_rest_equilibrium():
    """Eq. 11 with reading R23: the segregation weight is f_i^eq(rho, 0)/rho of
    the lattice equilibrium, which is w_i for the standard lattice; for the
    alpha-model at density ratio 10 it keeps the red populations of an
    interface cell at rest non-negative where w_i would drive them negative."""
    D = 2
    e, w, _, Minv = lat(D)
    import workloads
    aR, aB = workloads._alphas(2, 0.1, 1.0)
    cfg = _cfg(rhoR0=0.1, rhoB0=1.0, alphaR=aR, alphaB=aB, muR0=0.016, muB0=0.16)
    rR, rB = 0.05, 0.5
    fR = Minv @ ora.meq(2, rR, [0, 0, 0], aR)
    fB = Minv @ ora.meq(2, rB, [0, 0, 0], aB)
    z = np.zeros(3)
    g = np.array([0.4, 0.0, 0.0])
    fR2, fB2 = ora.collide_cell(cfg, D, fR, fB, z, z, z, z, g)
    assert fR2.min() >= 0 and fB2.min() >= 0
    # red momentum: beta (rR rB / rho) sum_i (feq0_i/rho) e_ix^2 with
    # sum_i feq0_i e_ix^2 = p = sum_k rho^k (c_s^k)^2 (App. A)
    rho = rR + rB
    p = rR * ora.cs2(2, aR) + rB * ora.cs2(2, aB)
    assert np.isclose((fR2 @ e[:, :2])[0], 0.7 * rR * rB / rho * p / rho, rtol=1e-10)
