"""Seeded synthetic workloads: parameter sets and initial fields.

This module is the only code shared by the CUDA path's tests/benchmark and
the CPU oracle.  It holds no arithmetic of the method itself: it converts the
dimensionless groups of the paper's test cases into lattice parameters and
draws initial fields (a circular / spherical droplet or bubble, uniform bulk
surfactant outside it, optional seeded perturbations).

Parameter keys (lattice units, delta_x = delta_t = 1):
  nx, ny, nz            grid (nz = 1: D2Q9, nz > 1: D3Q19)
  wall[3]               0 periodic / 1 half-way bounce-back walls per axis
  uw_lo, uw_hi          3x3 wall velocities (row = axis of the wall)
  rhoR0, rhoB0          pure-phase densities (red = droplet/bubble)
  muR0, muB0            pure-phase dynamic viscosities
  alphaR, alphaB        sound-speed parameters (light phase standard,
                        heavy phase from the density ratio, Eq. 42)
  sigma0, sigma_min_ratio, E0, psi_inf, beta
  eos (0 Langmuir, 1 linear), source (0 Eq. 22, 1 r_a psi_inf C),
  transport (1 solve the surfactant equations, 0 hold psi, C fixed)
  Ds, Db, ra, rd, g[3], sor_omega, eps_w, eps_n
  geometry: center[3], R, width, C0, psi0
"""
import math

import numpy as np

ALPHA_STD = {2: 4.0 / 9.0, 3: 1.0 / 3.0}


def _alphas(D, rhoR0, rhoB0):
    """Light phase standard; heavy phase alpha from Eq. 42 (equal pressure
    of the two pure phases at rest)."""
    a_std = ALPHA_STD[D]
    if rhoR0 <= rhoB0:
        gamma = rhoR0 / rhoB0
        return a_std, 1.0 - gamma * (1.0 - a_std)
    gamma = rhoB0 / rhoR0
    return 1.0 - gamma * (1.0 - a_std), a_std


def base(nx, ny, nz=1):
    D = 2 if nz == 1 else 3
    a = ALPHA_STD[D]
    return dict(
        nx=nx, ny=ny, nz=nz, wall=[0, 0, 0],
        uw_lo=[[0.0] * 3 for _ in range(3)], uw_hi=[[0.0] * 3 for _ in range(3)],
        rhoR0=1.0, rhoB0=1.0, muR0=0.1, muB0=0.1, alphaR=a, alphaB=a,
        sigma0=0.1, sigma_min_ratio=0.1, E0=0.5, psi_inf=1.0, beta=0.7,
        eos=0, source=0, transport=1,
        Ds=0.1, Db=0.1, ra=0.0, rd=0.0, g=[0.0, 0.0, 0.0],
        sor_omega=1.2, eps_w=1e-6, eps_n=1e-6,
        center=[(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0],
        R=min(nx, ny) / 4.0, width=3.0, C0=0.0, psi0=0.0,
    )


def droplet_adsorption_2d(n=128, R=25.0, C0=0.5):
    """2D stationary droplet adsorbing bulk surfactant (the 2D analogue of
    the paper's Sec. 3.1 test): D2Q9 n x n periodic, density and viscosity
    ratio 1 (rho = 1, mu = 0.1), sigma = 0.1, D_s = D_b = 0.1, E0 = 0.5,
    simple source j = r_a psi_inf C with r_a = 0.2, psi = 0 initially, bulk
    C0 outside the droplet, 0 inside."""
    c = base(n, n)
    c.update(R=float(R), C0=float(C0), ra=0.2, source=1, name="droplet_adsorption_2d")
    return c


def adsorption_octant_3d(R=20, C0=0.0005):
    """The paper's Sec. 3.1 test in 3D: one octant of a spherical droplet of
    radius R in a 5R x 5R x 5R D3Q19 domain, the droplet centred at the
    corner (-1/2, -1/2, -1/2) where three mirror planes meet (mirror planes
    half-way beyond both ends of every axis; the paper's far faces are
    periodic, which cannot coexist with the near mirror on one axis).
    rho = 1/1, mu = 0.1/0.1, sigma = 0.1, D_s = D_b = 0.1, E0 = 0.5, source
    j = r_a psi_inf C with r_a = 0.2 (adsorption only), psi = 0 initially,
    C = C0 = 0.0005 in the blue fluid."""
    n = int(round(5 * R))
    c = base(n, n, n)
    c.update(R=float(R), C0=float(C0), ra=0.2, source=1, wall=[2, 2, 2],
             center=[-0.5, -0.5, -0.5], name="adsorption_octant_3d")
    return c


def bubble_rise_3d(R=10, shape=(5, 5, 10), Eo=1.0, Mo=0.1, surfactant=True, Bi=10.0,
                   Pe=10.0, k=1.0, h=0.5, E0=0.5, C0=0.5, sigma0=0.004):
    """The paper's Sec. 3.4 test: a buoyant bubble (red, rho^R0 = 0.1) of
    radius R in a (shape[0] R) x (shape[1] R) x (shape[2] R) D3Q19 channel
    of liquid (rho^B0 = 1, mu^R0/mu^B0 = 0.1, sigma0 = 0.004), bounce-back
    walls on x and y, periodic z, gravity along -z, the bubble on the
    channel's axis at z = 2R.  g and mu^B0 from Eo and Mo as in
    bubble_rise_2d; with surfactant: E0 = 0.5, Pe_b = Pe_s = 10, k = 1,
    h = 0.5, Bi = 10, a clean interface at first (x_in = 0), C0 = 0.5 (not
    given in the paper); without, no surfactant at all (the clean case).
    The clean bubble's terminal velocity in an unbounded liquid is the
    Hadamard-Rybczynski velocity of Eq. 35 (bubble_rise_uth)."""
    nx, ny, nz = (int(round(q * R)) for q in shape)
    c = bubble_rise_2d(nx=nx, ny=ny, D_b=2.0 * R, Eo=Eo, Mo=Mo, Bi=Bi, Pe=Pe, k=k, h=h, E0=E0,
                       C0=C0, sigma0=sigma0)
    g = -c["g"][1]
    aR, aB = _alphas(3, c["rhoR0"], c["rhoB0"])
    c.update(nz=nz, wall=[1, 1, 0], g=[0.0, 0.0, -g], alphaR=aR, alphaB=aB,
             center=[(nx - 1) / 2.0, (ny - 1) / 2.0, 2.0 * R], name="bubble_rise_3d")
    if not surfactant:
        c.update(transport=0, C0=0.0, psi0=0.0, ra=0.0, rd=0.0)
    return c


def bubble_rise_uth(cfg):
    """Eq. 35: U_th = (2/3) g drho R^2 / mu^B0 (mu^B0 + mu^R0) / (2 mu^B0 + 3 mu^R0)."""
    g = abs(cfg["g"][2])
    drho = cfg["rhoB0"] - cfg["rhoR0"]
    mB, mR = cfg["muB0"], cfg["muR0"]
    return 2.0 / 3.0 * g * drho * cfg["R"] ** 2 / mB * (mB + mR) / (2 * mB + 3 * mR)


def migration_3d(R=10, shape=(5, 5, 10), sigma0=0.001, E0=0.5):
    """The paper's Sec. 3.2 test: a droplet of radius R in an
    (shape[0] R) x (shape[1] R) x (shape[2] R) D3Q19 box (5R x 5R x 10R or
    10R x 10R x 10R), bounce-back walls on x and y, periodic z, rho = 1/1,
    mu = 0.1/0.1, linear equation of state sigma = sigma0 (1 - E0 psi/psi_inf)
    with sigma0 = 0.001, E0 = 0.5, and insoluble surfactant held at
    psi = psi_inf (z + 1/2) / L_z (Eq. 31; x_in = 0.5 at the droplet's
    centre): no surfactant transport.  The Marangoni stress drives the
    droplet towards +z; its terminal velocity in an unbounded fluid is the
    YGB velocity of Eq. 32 (migration_ygb)."""
    nx, ny, nz = (int(round(k * R)) for k in shape)
    c = base(nx, ny, nz)
    c.update(R=float(R), wall=[1, 1, 0], eos=1, sigma0=sigma0, E0=E0, psi_inf=1.0,
             transport=0, C0=0.0, psi_profile="linear_z", name="migration_3d")
    return c


def migration_ygb(cfg):
    """Eq. 32: U_YGB = 2 sigma0 E0 R / (L_z (6 mu^R0 + 9 mu^B0))."""
    return 2 * cfg["sigma0"] * cfg["E0"] * cfg["R"] / (
        cfg["nz"] * (6 * cfg["muR0"] + 9 * cfg["muB0"]))


def adsorption_analytic(cfg, t, r):
    """Short-time sharp-interface solutions of Sec. 3.1 for a sphere:
    (C(r, t)/C0 of Eq. 29, psi(t)/psi_inf of Eq. 30), with D the bulk
    diffusivity, m = r_a psi_inf / D, a = sqrt(pi D), eta = a (1 + R m)/R.
    Eq. 29 is read with the product sqrt(pi D t)(1 + R m) divided by R in its
    denominator (as printed it adds a length to 1; with the division the
    interface value tends to the steady 1/(1 + R m), and Eq. 30's long-time
    slope r_a C0/(1 + R m) follows)."""
    from math import erfc, log, pi, sqrt
    D, R, ra, pinf, C0 = cfg["Db"], cfg["R"], cfg["ra"], cfg["psi_inf"], cfg["C0"]
    m = ra * pinf / D
    a = sqrt(pi * D)
    eta = a * (1 + R * m) / R
    s = sqrt(pi * D * t)
    amp = (m * s) / (1 + s * (1 + R * m) / R)
    c = [1 - amp * (R / ri) * erfc((ri - R) / (2 * sqrt(D * t))) for ri in r]
    psi = cfg["psi0"] / pinf + ra * C0 * (
        t - (a * m / eta ** 3) * (eta ** 2 * t - 2 * eta * sqrt(t) + 2 * log(1 + eta * sqrt(t))))
    return np.array(c), psi


def bubble_rise_2d(nx=256, ny=1024, D_b=64.0, Eo=10.0, Mo=0.1, Bi=1.0, Pe=10.0,
                   k=1.0, h=0.5, E0=0.5, C0=0.5, sigma0=0.004, rho_ratio=10.0,
                   mu_ratio=10.0, y0=None):
    """2D buoyant bubble in a walled channel (2D version of Sec. 3.4):
    D2Q9 nx x ny, bounce-back walls at x = -1/2 and nx - 1/2, periodic in y,
    gravity along -y.  Lattice parameters from the dimensionless groups:
      g   = Eo sigma0 / (drho (2R)^2)                  (Eotvos number)
      muB = (Mo rhoB0^2 sigma0^3 / (drho g))^(1/4)     (Morton number)
      U_ref = sqrt(2 R g), t_ref = 2R / U_ref          (tau of Sec. 3.4)
      r_d = Bi / t_ref, D_s = D_b = U_ref 2R / Pe, r_a = k r_d / C0
      psi_inf = h C0 R (1 + k) / k   (h of Sec. 3.3 with psi0 taken as the
                                      equilibrium coverage psi_inf k/(1+k))."""
    R = D_b / 2.0
    rhoB0, rhoR0 = 1.0, 1.0 / rho_ratio
    drho = rhoB0 - rhoR0
    g = Eo * sigma0 / (drho * (2 * R) ** 2)
    muB = (Mo * rhoB0 ** 2 * sigma0 ** 3 / (drho * g)) ** 0.25
    U = math.sqrt(2 * R * g)
    t_ref = 2 * R / U
    rd = Bi / t_ref
    Dd = U * 2 * R / Pe
    c = base(nx, ny)
    aR, aB = _alphas(2, rhoR0, rhoB0)
    c.update(
        name="bubble_rise_2d", wall=[1, 0, 0], rhoR0=rhoR0, rhoB0=rhoB0,
        muB0=muB, muR0=muB / mu_ratio, alphaR=aR, alphaB=aB,
        sigma0=sigma0, E0=E0, psi_inf=h * C0 * R * (1 + k) / k,
        Ds=Dd, Db=Dd, rd=rd, ra=k * rd / C0, source=0,
        g=[0.0, -g, 0.0], R=R, C0=C0, psi0=0.0,
        center=[(nx - 1) / 2.0, (2.0 * R if y0 is None else y0), 0.0],
        Eo=Eo, Mo=Mo, Bi=Bi, Pe=Pe, U_ref=U, t_ref=t_ref,
    )
    return c


def bubble_array_2d(n=4096, k=16, **kw):
    """The bubble rise's physics (bubble_rise_2d: D = 64, Eo = 10, density
    ratio 10, walls on x, periodic y) on an n x n grid holding a k x k array
    of bubbles, one at the centre of each (n/k) x (n/k) block: at 4096 x 4096
    with 16 x 16 bubbles, 16.8 M cells and about 3 GB of FP32 state, far
    beyond the L2 (the single 256 x 1024 bubble fits in it).  The array is
    periodic in y with period n/k, so the exact solution is too."""
    c = bubble_rise_2d(nx=n, ny=n, **kw)
    s = n / k
    c.update(name="bubble_array_2d", array=[k, k, s, s],
             center=[s / 2.0 - 0.5, s / 2.0 - 0.5, 0.0])
    return c


SWEEP_WIDTHS = (64, 96, 128, 192, 256)


def sweep_point(rng, vary_surfactant=True):
    """One point of the batched bubble-rise sweep: Eo log-uniform in [1, 50],
    Bi log-uniform in [0.01, 10], channel width uniform in SWEEP_WIDTHS
    (confinement D / width with D = 32), height uniform in [512, 1024];
    with vary_surfactant the elasticity E0 (uniform [0.2, 0.8]) and the bulk
    concentration C0 (uniform [0.25, 1]) vary too (the surrogate's inputs),
    else they keep the bubble-rise values 0.5 / 0.5."""
    Eo = float(np.exp(rng.uniform(np.log(1.0), np.log(50.0))))
    Bi = float(np.exp(rng.uniform(np.log(0.01), np.log(10.0))))
    width = int(rng.choice(SWEEP_WIDTHS))
    height = int(rng.integers(512, 1025))
    E0 = float(rng.uniform(0.2, 0.8)) if vary_surfactant else 0.5
    C0 = float(rng.uniform(0.25, 1.0)) if vary_surfactant else 0.5
    return dict(Eo=Eo, Bi=Bi, width=width, height=height, E0=E0, C0=C0)


def sweep_instance(pt, D_b=32.0):
    """The bubble-rise instance of a sweep point (density ratio 10,
    viscosity ratio 10, Mo = 0.1, Pe = 10, k = 1, h = 0.5)."""
    c = bubble_rise_2d(nx=pt["width"], ny=pt["height"], D_b=D_b, Eo=pt["Eo"], Bi=pt["Bi"],
                       E0=pt["E0"], C0=pt["C0"])
    c["name"] = "sweep_bubble_2d"
    c["sweep_point"] = dict(pt)
    return c


def bubble_sweep_2d(n=64, seed=0, vary_surfactant=True):
    """n seeded sweep instances (the batched configuration: 64 instances of
    widths 64-256 and heights 512-1024, D = 32)."""
    rng = np.random.default_rng(seed)
    return [sweep_instance(sweep_point(rng, vary_surfactant)) for _ in range(n)]


# width of the steady colour profile tanh(d / W) that the recolouring of
# Eq. 11 with beta = 0.7 maintains (measured on a flat interface, D2Q9 and
# D3Q19 alike: 1.40 lattice units)
EQ_WIDTH = 1.4


def shear_droplet_3d(nx=256, ny=128, nz=128, R=24.0, Ca=0.2, Re=1.0, lam=1.0, C0=0.5,
                     E0=0.3, sigma0=5e-4, x_in=0.5, h=0.5, Bi=1.0, Pe_s=10.0, Pe_b=10.0,
                     width=EQ_WIDTH):
    """3D surfactant-laden droplet in simple shear (the 3D analogue of the
    paper's Sec. 3.3 set-up): D3Q19 nx x ny x nz, half-way bounce-back walls
    at z = -1/2 and nz - 1/2 moving with -u_w and +u_w along x, periodic in
    x and y; droplet of radius R at the centre, density ratio 1.
    Dimensionless groups of Sec. 3.3 (L = R, U = u_w / 2, shear rate
    2 u_w / H with H = nz):
      Re = rho U R / mu and Ca = mu U / sigma0 give mu = sqrt(Ca Re sigma0 R)
      (rho = 1) and U = Ca sigma0 / mu;
      Pe_s = U R / D_s, Pe_b = U R / D_b;  Bi = r_d / shear rate;
      x_in = psi0 / psi_inf;  h = psi0 / (C0 R);  k = r_a C0 / r_d, with
      no initial mass transfer (j = 0 at psi0, C0) so that k = x_in/(1-x_in).
    psi starts uniform at its Langmuir equilibrium psi0 (Eq. 22 with j = 0),
    C = C0 in the liquid.  The colour profile starts at the recolouring's
    own steady width (EQ_WIDTH): Eqs. 20-21 conserve |grad rhoN| psi and
    (1 - rhoN) C, so an initial profile wider than the steady one, sharpening
    in the first hundred steps, would divide the surfactant already in its
    flanks by weights that shrink towards zero (psi and C then grow without
    bound inside a small droplet)."""
    mu = math.sqrt(Ca * Re * sigma0 * R)
    U = Ca * sigma0 / mu
    uw = 2.0 * U
    rate = 2.0 * uw / nz
    psi0 = h * C0 * R
    k = x_in / (1.0 - x_in)
    rd = Bi * rate
    c = base(nx, ny, nz)
    c.update(
        name="shear_droplet_3d", wall=[0, 0, 1],
        uw_lo=[[0.0] * 3, [0.0] * 3, [-uw, 0.0, 0.0]],
        uw_hi=[[0.0] * 3, [0.0] * 3, [uw, 0.0, 0.0]],
        muR0=lam * mu, muB0=mu, sigma0=sigma0, E0=E0, psi_inf=psi0 / x_in,
        Ds=U * R / Pe_s, Db=U * R / Pe_b, rd=rd, ra=k * rd / C0, source=0,
        R=float(R), C0=C0, psi0=psi0, psi_profile="uniform", width=float(width),
        Ca=Ca, Re=Re, U_ref=U, shear_rate=rate,
    )
    return c


def initial_fields(cfg, seed=None, noise=0.0, u0=None):
    """Colour field phi = tanh((R - r)/width) (red inside), psi = psi0 times
    the interface indicator (1 - phi^2) (or psi0 everywhere when
    cfg["psi_profile"] == "uniform", psi_inf (z + 1/2)/nz when it is
    "linear_z"), C = C0 (1 - phi)/2 (bulk surfactant
    in the blue fluid only).  With a seed, psi and C receive multiplicative
    uniform noise of relative amplitude `noise` and u gets an additive field
    of amplitude `u0` (both break mirror symmetry for parity tests).  With
    cfg["array"] = [kx, ky, sx, sy] the distance r is to the centre of the
    cell's own sx x sy block (an array of bubbles)."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg.get("nz", 1)
    cx, cy, cz = cfg["center"]
    if "array" in cfg:  # a bubble at the centre of every (sx x sy) block (2D)
        _, _, sx, sy = cfg["array"]
        dx = np.mod(np.arange(nx, dtype=np.float64), sx) - cx
        dy = np.mod(np.arange(ny, dtype=np.float64), sy) - cy
        r = np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2)[None]
    else:
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + ((z - cz) ** 2 if nz > 1 else 0.0))
    phi = np.tanh((cfg["R"] - r) / cfg["width"])
    if cfg.get("psi_profile") == "uniform":
        psi = np.full_like(phi, cfg["psi0"])
    elif cfg.get("psi_profile") == "linear_z":  # Eq. 31, every cell
        zz = (np.arange(nz, dtype=np.float64) + 0.5) / nz
        psi = cfg["psi_inf"] * np.broadcast_to(zz[:, None, None], phi.shape).copy()
    else:
        psi = cfg["psi0"] * (1.0 - phi ** 2)
    C = cfg["C0"] * 0.5 * (1.0 - phi)
    u = np.zeros((3, nz, ny, nx))
    if seed is not None:
        rng = np.random.default_rng(seed)
        if noise:
            psi = psi * (1.0 + noise * rng.uniform(-1, 1, psi.shape))
            C = C * (1.0 + noise * rng.uniform(-1, 1, C.shape))
        if u0:
            D = 2 if nz == 1 else 3
            u[:D] = u0 * rng.uniform(-1, 1, (D, nz, ny, nx))
    return dict(phi=phi, psi=psi, C=C, u=u)
