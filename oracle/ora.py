"""ctypes binding of the FP64 CPU oracle (``oracle/liboracle.so``).

Test infrastructure only.  Fields are numpy float64 arrays shaped
``(nz, ny, nx)``; vector fields ``(3, nz, ny, nx)``; populations
``(Q, nz, ny, nx)``.
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None


class OraParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("wall", C.c_int * 3),
        ("uw_lo", (C.c_double * 3) * 3), ("uw_hi", (C.c_double * 3) * 3),
        ("rhoR0", C.c_double), ("rhoB0", C.c_double),
        ("muR0", C.c_double), ("muB0", C.c_double),
        ("alphaR", C.c_double), ("alphaB", C.c_double),
        ("sigma0", C.c_double), ("sigma_min_ratio", C.c_double),
        ("E0", C.c_double), ("psi_inf", C.c_double), ("beta", C.c_double),
        ("eos", C.c_int), ("source", C.c_int), ("transport", C.c_int),
        ("Ds", C.c_double), ("Db", C.c_double),
        ("ra", C.c_double), ("rd", C.c_double),
        ("g", C.c_double * 3),
        ("sor_omega", C.c_double), ("sor_tol", C.c_double),
        ("sor_max_iter", C.c_int),
        ("eps_w", C.c_double), ("eps_n", C.c_double),
    ]


class OraDiag(C.Structure):
    _fields_ = [
        ("mass_R", C.c_double), ("mass_B", C.c_double),
        ("surf_total", C.c_double), ("surf_pre_rescale", C.c_double),
        ("rescale_factor", C.c_double),
        ("U", C.c_double * 3), ("centroid", C.c_double * 3),
        ("aspect_ratio", C.c_double),
        ("psi_av", C.c_double), ("psi_min", C.c_double), ("psi_max", C.c_double),
        ("umax", C.c_double), ("Re", C.c_double),
        ("sor_iters_psi", C.c_int), ("sor_iters_C", C.c_int),
        ("step", C.c_longlong),
    ]


_DP = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        L.ora_create.restype = C.c_void_p
        L.ora_create.argtypes = [C.POINTER(OraParams)]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_init_fields.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP]
        L.ora_step.argtypes = [C.c_void_p, C.c_int]
        L.ora_get_fields.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP, _DP]
        L.ora_diagnostics.argtypes = [C.c_void_p, C.POINTER(OraDiag)]
        L.ora_get_pops.argtypes = [C.c_void_p, _DP, _DP]
        L.ora_set_pops.argtypes = [C.c_void_p, _DP, _DP]
        L.ora_set_surfactant.argtypes = [C.c_void_p, _DP, _DP]
        L.ora_step_count.restype = C.c_longlong
        L.ora_step_count.argtypes = [C.c_void_p]
        L.ora_threads.restype = C.c_int
        L.ora_threads.argtypes = [C.c_int]
        L.ora_set_ends.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
        L.ora_phase.argtypes = [C.c_void_p, C.c_int]
        _D = C.POINTER(C.c_double)
        L.ora_sor_rows.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, _D, _D]
        L.ora_surf_rows.argtypes = [C.c_void_p, C.c_int, C.c_int, _D]
        L.ora_finish.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int]
        L.ora_set_M0.argtypes = [C.c_void_p, C.c_double]
        L.ora_field.restype = _D
        L.ora_field.argtypes = [C.c_void_p, C.c_char_p]
        L.ora_macro.argtypes = [C.c_void_p] + [_DP] * 10
        L.ora_lattice.argtypes = [C.c_int, C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), _DP, _DP, _DP]
        L.ora_meq.argtypes = [C.c_int, C.c_double, _DP, C.c_double, _DP]
        L.ora_corr.argtypes = [C.c_int, _DP, _DP]
        L.ora_relax.argtypes = [C.c_int, C.c_double, _DP]
        L.ora_forcing.argtypes = [C.c_int, _DP, _DP, _DP]
        L.ora_cs2.restype = C.c_double
        L.ora_cs2.argtypes = [C.c_int, C.c_double]
        L.ora_collide_cell.argtypes = [C.POINTER(OraParams), C.c_int] + [_DP] * 9
        L.ora_eos.argtypes = [C.POINTER(OraParams), C.c_double, _DP, _DP]
        L.ora_cmc.restype = C.c_double
        L.ora_cmc.argtypes = [C.POINTER(OraParams)]
        L.ora_iso_grad.argtypes = [C.c_void_p, _DP, _DP]
        L.ora_weno_div.argtypes = [C.c_void_p, _DP, _DP, _DP]
        L.ora_diffuse.argtypes = [C.c_void_p, _DP, _DP, _DP]
        L.ora_sor.argtypes = [C.c_void_p, _DP, C.c_double, _DP, _DP]
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _vec(v, n=3):
    return np.ascontiguousarray(np.resize(np.asarray(v, np.float64), n))


def make_params(cfg: dict) -> OraParams:
    """Fill the oracle's parameter struct from a workload parameter dict."""
    p = OraParams()
    p.nx, p.ny, p.nz = cfg["nx"], cfg["ny"], cfg.get("nz", 1)
    for a in range(3):
        p.wall[a] = int(cfg.get("wall", (0, 0, 0))[a])
        for b in range(3):
            p.uw_lo[a][b] = cfg.get("uw_lo", [[0] * 3] * 3)[a][b]
            p.uw_hi[a][b] = cfg.get("uw_hi", [[0] * 3] * 3)[a][b]
    for k in ("rhoR0", "rhoB0", "muR0", "muB0", "alphaR", "alphaB", "sigma0",
              "sigma_min_ratio", "E0", "psi_inf", "beta", "Ds", "Db", "ra",
              "rd", "sor_omega", "eps_w", "eps_n"):
        setattr(p, k, float(cfg[k]))
    p.eos, p.source, p.transport = int(cfg["eos"]), int(cfg["source"]), int(cfg["transport"])
    for a in range(3):
        p.g[a] = float(cfg.get("g", (0, 0, 0))[a])
    p.sor_tol = float(cfg.get("oracle_sor_tol", 1e-13))
    p.sor_max_iter = int(cfg.get("oracle_sor_max_iter", 10000))
    return p


def threads(n=0):
    """Host threads of the oracle's independent cell loops (OpenMP): n > 0
    sets the count for the process; returns the count in use."""
    return int(lib().ora_threads(int(n)))


class Oracle:
    """One oracle simulation context."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self.p = make_params(cfg)
        self.shape = (self.p.nz, self.p.ny, self.p.nx)
        self.N = int(np.prod(self.shape))
        self.D = 2 if self.p.nz == 1 else 3
        self.Q = 9 if self.D == 2 else 19
        self.h = lib().ora_create(C.byref(self.p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_destroy(self.h)
            self.h = None

    def _f(self, x, comps=None):
        if x is None:
            return None
        shape = self.shape if comps is None else (comps,) + self.shape
        return np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), shape))

    def init_fields(self, phi, psi, C_, u=None):
        self._keep = [self._f(phi), self._f(psi), self._f(C_), self._f(u, 3)]
        r = lib().ora_init_fields(self.h, *[_p(a) for a in self._keep])
        assert r == 0

    def set_surfactant(self, psi, C_):
        a, b = self._f(psi), self._f(C_)
        assert lib().ora_set_surfactant(self.h, _p(a), _p(b)) == 0

    def step(self, n=1):
        r = lib().ora_step(self.h, int(n))
        if r != 0:
            raise RuntimeError(f"oracle step failed ({r})")

    @property
    def step_count(self):
        return lib().ora_step_count(self.h)

    def fields(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        phi, psi, C_ = (np.empty(self.shape) for _ in range(3))
        lib().ora_get_fields(self.h, _p(rho), _p(u), _p(phi), _p(psi), _p(C_))
        return dict(rho=rho, u=u, phi=phi, psi=psi, C=C_)

    def pops(self):
        fR = np.empty((self.Q,) + self.shape)
        fB = np.empty((self.Q,) + self.shape)
        lib().ora_get_pops(self.h, _p(fR), _p(fB))
        return fR, fB

    def set_pops(self, fR, fB):
        a, b = self._f(fR, self.Q), self._f(fB, self.Q)
        lib().ora_set_pops(self.h, _p(a), _p(b))

    def macro(self):
        out = dict(rhoR=np.empty(self.shape), rhoB=np.empty(self.shape),
                   rhoN=np.empty(self.shape), g=np.empty((3,) + self.shape),
                   a=np.empty(self.shape), kappa=np.empty(self.shape),
                   F=np.empty((3,) + self.shape), u=np.empty((3,) + self.shape),
                   S=np.empty(self.shape), B=np.empty(self.shape))
        lib().ora_macro(self.h, *[_p(out[k]) for k in
                                  ("rhoR", "rhoB", "rhoN", "g", "a", "kappa",
                                   "F", "u", "S", "B")])
        return out

    def diagnostics(self):
        d = OraDiag()
        lib().ora_diagnostics(self.h, C.byref(d))
        return {k: (list(getattr(d, k)) if k in ("U", "centroid") else getattr(d, k))
                for k, _ in OraDiag._fields_}

    # finite-difference building blocks on this context's grid
    def iso_grad(self, x):
        x = self._f(x)
        g = np.empty((3,) + self.shape)
        lib().ora_iso_grad(self.h, _p(x), _p(g))
        return g

    def weno_div(self, Psi, u):
        Psi, u = self._f(Psi, 3), self._f(u, 3)
        out = np.empty(self.shape)
        lib().ora_weno_div(self.h, _p(Psi), _p(u), _p(out))
        return out

    def diffuse(self, w, x):
        w, x = self._f(w), self._f(x)
        out = np.empty(self.shape)
        lib().ora_diffuse(self.h, _p(w), _p(x), _p(out))
        return out

    def sor(self, w, h, rhs, x0):
        w, rhs = self._f(w), self._f(rhs)
        x = self._f(x0).copy()
        it = lib().ora_sor(self.h, _p(w), float(h), _p(rhs), _p(x))
        return x, it


# ---- cell-level building blocks -------------------------------------------
def lattice(D):
    q = C.c_int()
    Q = 9 if D == 2 else 19
    e = (C.c_int * (3 * Q))()
    w, M, Minv = np.empty(Q), np.empty((Q, Q)), np.empty((Q, Q))
    assert lib().ora_lattice(D, C.byref(q), e, _p(w), _p(M), _p(Minv)) == 0
    return np.array(e[:], dtype=int).reshape(Q, 3), w, M, Minv


def meq(D, rho, u, alpha):
    Q = 9 if D == 2 else 19
    m = np.empty(Q)
    lib().ora_meq(D, rho, _p(_vec(u)), alpha, _p(m))
    return m


def corr(D, Qv):
    Q = 9 if D == 2 else 19
    c = np.empty(Q)
    lib().ora_corr(D, _p(_vec(Qv)), _p(c))
    return c


def relax(D, sv):
    Q = 9 if D == 2 else 19
    S = np.empty(Q)
    lib().ora_relax(D, sv, _p(S))
    return S


def forcing(D, u, F):
    Q = 9 if D == 2 else 19
    out = np.empty(Q)
    lib().ora_forcing(D, _p(_vec(u)), _p(_vec(F)), _p(out))
    return out


def cs2(D, alpha):
    return lib().ora_cs2(D, alpha)


def collide_cell(cfg, D, fR, fB, u, F, dRu, dBu, g):
    p = make_params(cfg)
    Q = 9 if D == 2 else 19
    fR2, fB2 = np.empty(Q), np.empty(Q)
    args = [np.ascontiguousarray(np.asarray(fR, np.float64)),
            np.ascontiguousarray(np.asarray(fB, np.float64)),
            _vec(u), _vec(F), _vec(dRu), _vec(dBu), _vec(g)]
    lib().ora_collide_cell(C.byref(p), D, *[_p(a) for a in args], _p(fR2), _p(fB2))
    return fR2, fB2


def eos(cfg, psi):
    p = make_params(cfg)
    s, m = C.c_double(), C.c_double()
    lib().ora_eos(C.byref(p), float(psi), C.byref(s), C.byref(m))
    return s.value, m.value


def cmc(cfg):
    return lib().ora_cmc(C.byref(make_params(cfg)))
