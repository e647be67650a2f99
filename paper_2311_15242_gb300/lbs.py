"""Python binding of the C ABI in ``include/lbs.h`` (``liblbs.so``).

Argument marshalling only: every step of the coupled update runs in the CUDA
kernels of the library.  PyTorch supplies the device workspace and the CUDA
stream.  There is no CPU fallback: loading fails loudly when the library or
a CUDA device is missing.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

LBS_OK, LBS_EINVAL, LBS_ENOMEM, LBS_ECUDA = 0, -1, -2, -3
LBS_ENOCONV, LBS_EDIVERGED, LBS_ETIMEOUT, LBS_EBOUNDS = -4, -5, -6, -7
LBS_F64, LBS_F32, LBS_F16, LBS_BF16 = 0, 1, 2, 3
STORAGE = {"f64": LBS_F64, "f32": LBS_F32, "f16": LBS_F16, "bf16": LBS_BF16}

EXPORTS = ("lbs_params_default", "lbs_workspace_bytes", "lbs_create",
           "lbs_init_fields", "lbs_step", "lbs_sync", "lbs_get_fields",
           "lbs_get_macro", "lbs_diagnostics", "lbs_profile", "lbs_kernel_times", "lbs_set_graph",
           "lbs_step_kernel_count", "lbs_set_sor_tile", "lbs_set_sor_persistent", "lbs_set_sor_wait_limit",
           "lbs_step_result", "lbs_save_state", "lbs_load_state",
           "lbs_surfactant_total_static",
           "lbs_destroy",
           "lbs_last_error", "lbs_batch_workspace_bytes", "lbs_batch_create",
           "lbs_batch_init_fields", "lbs_batch_set_tiles", "lbs_batch_step", "lbs_batch_sync",
           "lbs_batch_get_fields", "lbs_batch_diagnostics", "lbs_batch_set_graph",
           "lbs_batch_step_kernel_count", "lbs_batch_status", "lbs_batch_set_active",
           "lbs_batch_destroy", "lbs_batch_last_error",
           "lbs_mlp_create", "lbs_mlp_param_count", "lbs_mlp_init", "lbs_mlp_set_params",
           "lbs_mlp_get_params", "lbs_mlp_forward", "lbs_mlp_gradient", "lbs_mlp_set_grad",
           "lbs_mlp_adam_step", "lbs_mlp_set_data", "lbs_mlp_train", "lbs_mlp_predict",
           "lbs_mlp_destroy", "lbs_mlp_last_error")
KERNEL_GROUPS = ("force", "fd", "collide", "stream", "grad", "sor", "surf")


class LbsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbs error {code}: {msg}")
        self.code = code


class LbsParams(C.Structure):
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
        ("Ds", C.c_double), ("Db", C.c_double), ("ra", C.c_double), ("rd", C.c_double),
        ("g", C.c_double * 3),
        ("sor_omega", C.c_double), ("sor_tol", C.c_double), ("sor_max_iter", C.c_int),
        ("eps_w", C.c_double), ("eps_n", C.c_double),
    ]


class LbsDiag(C.Structure):
    _fields_ = [
        ("mass_R", C.c_double), ("mass_B", C.c_double),
        ("surf_total", C.c_double), ("surf_pre_rescale", C.c_double),
        ("rescale_factor", C.c_double),
        ("U", C.c_double * 3), ("centroid", C.c_double * 3),
        ("aspect_ratio", C.c_double),
        ("psi_av", C.c_double), ("psi_min", C.c_double), ("psi_max", C.c_double),
        ("umax", C.c_double), ("Re", C.c_double),
        ("sor_iters_psi", C.c_int), ("sor_iters_C", C.c_int), ("sor_rounds", C.c_int),
        ("step", C.c_longlong),
        ("deformation", C.c_double), ("inclination", C.c_double),
    ]


_lib = None
_DP = C.POINTER(C.c_double)


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbs.so (building it in-tree if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library missing: {path}")
    L = C.CDLL(path)
    L.lbs_params_default.argtypes = [C.POINTER(LbsParams), C.c_int, C.c_int, C.c_int]
    L.lbs_workspace_bytes.restype = C.c_size_t
    L.lbs_workspace_bytes.argtypes = [C.POINTER(LbsParams), C.c_int]
    L.lbs_create.argtypes = [C.POINTER(LbsParams), C.c_int, C.c_void_p, C.c_void_p,
                             C.c_size_t, C.POINTER(C.c_void_p)]
    L.lbs_init_fields.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP]
    L.lbs_step.argtypes = [C.c_void_p, C.c_int]
    L.lbs_sync.argtypes = [C.c_void_p]
    L.lbs_get_fields.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP, _DP]
    L.lbs_diagnostics.argtypes = [C.c_void_p, C.POINTER(LbsDiag)]
    L.lbs_profile.argtypes = [C.c_void_p, C.c_int]
    L.lbs_kernel_times.argtypes = [C.c_void_p, _DP, C.c_int]
    L.lbs_step_kernel_count.argtypes = [C.c_void_p]
    L.lbs_set_graph.argtypes = [C.c_void_p, C.c_int]
    L.lbs_set_sor_tile.argtypes = [C.c_void_p, C.c_int]
    L.lbs_set_sor_persistent.argtypes = [C.c_void_p, C.c_int]
    L.lbs_set_sor_wait_limit.argtypes = [C.c_void_p, C.c_longlong]
    L.lbs_step_result.argtypes = [C.c_void_p, _DP]
    L.lbs_save_state.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]
    L.lbs_load_state.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
    L.lbs_get_macro.argtypes = [C.c_void_p] + [_DP] * 6
    L.lbs_surfactant_total_static.argtypes = [C.c_int] + [C.c_void_p] * 4 + [C.c_int] * 4 + [
        C.c_double, C.c_void_p, C.c_void_p]
    L.lbs_destroy.argtypes = [C.c_void_p]
    L.lbs_last_error.restype = C.c_char_p
    L.lbs_last_error.argtypes = [C.c_void_p]
    L.lbs_batch_workspace_bytes.restype = C.c_size_t
    L.lbs_batch_workspace_bytes.argtypes = [C.POINTER(LbsParams), C.c_int, C.c_int]
    L.lbs_batch_create.argtypes = [C.POINTER(LbsParams), C.c_int, C.c_int, C.c_void_p,
                                   C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]
    L.lbs_batch_init_fields.argtypes = [C.c_void_p, C.c_int, _DP, _DP, _DP, _DP]
    L.lbs_batch_set_tiles.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.lbs_batch_step.argtypes = [C.c_void_p, C.c_int]
    L.lbs_batch_sync.argtypes = [C.c_void_p]
    L.lbs_batch_get_fields.argtypes = [C.c_void_p, C.c_int, _DP, _DP, _DP, _DP, _DP]
    L.lbs_batch_diagnostics.argtypes = [C.c_void_p, C.POINTER(LbsDiag)]
    L.lbs_batch_set_graph.argtypes = [C.c_void_p, C.c_int]
    L.lbs_batch_step_kernel_count.argtypes = [C.c_void_p]
    L.lbs_batch_status.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    _FP = C.POINTER(C.c_float)
    L.lbs_mlp_create.argtypes = [C.c_int] * 6 + [C.c_void_p, C.POINTER(C.c_void_p)]
    L.lbs_mlp_param_count.argtypes = [C.c_void_p]
    L.lbs_mlp_init.argtypes = [C.c_void_p, C.c_ulonglong]
    L.lbs_mlp_set_params.argtypes = [C.c_void_p, _FP]
    L.lbs_mlp_get_params.argtypes = [C.c_void_p, _FP]
    L.lbs_mlp_forward.argtypes = [C.c_void_p, _FP, C.c_int, C.c_int, _FP]
    L.lbs_mlp_gradient.argtypes = [C.c_void_p, _FP, _FP, C.c_int, _FP, _DP]
    L.lbs_mlp_set_grad.argtypes = [C.c_void_p, _FP]
    L.lbs_mlp_adam_step.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float]
    L.lbs_mlp_set_data.argtypes = [C.c_void_p, _FP, _FP, C.c_int]
    L.lbs_mlp_train.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                                C.c_float, C.c_ulonglong, _DP]
    L.lbs_mlp_predict.argtypes = [C.c_void_p, _FP, C.c_int, C.c_int, _FP, _FP]
    L.lbs_mlp_destroy.argtypes = [C.c_void_p]
    L.lbs_mlp_last_error.restype = C.c_char_p
    L.lbs_mlp_last_error.argtypes = [C.c_void_p]
    L.lbs_batch_set_active.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.lbs_batch_destroy.argtypes = [C.c_void_p]
    L.lbs_batch_last_error.restype = C.c_char_p
    L.lbs_batch_last_error.argtypes = [C.c_void_p]
    _lib = L
    return L


def params_from(cfg: dict, storage: int) -> LbsParams:
    """Marshal a workload parameter dict into the ABI's parameter struct."""
    p = LbsParams()
    load().lbs_params_default(C.byref(p), int(cfg["nx"]), int(cfg["ny"]), int(cfg.get("nz", 1)))
    for a in range(3):
        p.wall[a] = int(cfg.get("wall", (0, 0, 0))[a])
        for b in range(3):
            p.uw_lo[a][b] = float(cfg.get("uw_lo", [[0] * 3] * 3)[a][b])
            p.uw_hi[a][b] = float(cfg.get("uw_hi", [[0] * 3] * 3)[a][b])
        p.g[a] = float(cfg.get("g", (0, 0, 0))[a])
    for k in ("rhoR0", "rhoB0", "muR0", "muB0", "alphaR", "alphaB", "sigma0",
              "sigma_min_ratio", "E0", "psi_inf", "beta", "Ds", "Db", "ra", "rd",
              "sor_omega", "eps_w", "eps_n"):
        if k in cfg:
            setattr(p, k, float(cfg[k]))
    for k in ("eos", "source", "transport"):
        if k in cfg:
            setattr(p, k, int(cfg[k]))
    p.sor_tol = float(cfg.get("sor_tol", 1e-13 if storage == LBS_F64 else 5e-7))
    p.sor_max_iter = int(cfg.get("sor_max_iter", 64 if storage == LBS_F64 else 48))
    return p


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


class Solver:
    """One solver context on the current CUDA device.

    The device workspace is a torch uint8 tensor and the work is queued on a
    torch CUDA stream (both borrowed by the library)."""

    def __init__(self, cfg: dict, storage="f32", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.L = load()
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.p = params_from(cfg, self.storage)
        self.shape = (self.p.nz, self.p.ny, self.p.nx)
        self.N = int(np.prod(self.shape))
        nbytes = self.L.lbs_workspace_bytes(C.byref(self.p), self.storage)
        if nbytes == 0:
            raise LbsError(LBS_EINVAL, "invalid parameters")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        # a stream of its own: the step graph is captured on it, which the
        # legacy default stream does not allow
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        r = self.L.lbs_create(C.byref(self.p), self.storage, C.c_void_p(self.stream.cuda_stream),
                              C.c_void_p(aligned), nbytes, C.byref(h))
        self.h = h
        self._check(r)

    def _check(self, r):
        if r != LBS_OK:
            msg = self.L.lbs_last_error(self.h).decode() if self.h else "?"
            raise LbsError(r, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.lbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f(self, x, comps=None):
        if x is None:
            return None
        shape = self.shape if comps is None else (comps,) + self.shape
        return np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), shape))

    def init_fields(self, phi, psi=None, C_=None, u=None):
        arrs = [self._f(phi), self._f(psi), self._f(C_), self._f(u, 3)]
        self._check(self.L.lbs_init_fields(self.h, *[_dp(a) for a in arrs]))

    def step(self, n=1):
        self._check(self.L.lbs_step(self.h, int(n)))

    def sync(self):
        self._check(self.L.lbs_sync(self.h))

    def fields(self, out=None):
        """rho, u (3 components), phi, psi, C as float64 arrays of the grid's
        shape; into the caller's arrays when `out` holds them (page-locked
        ones make the copy faster), else into new ones."""
        if out is None:
            out = dict(rho=np.empty(self.shape), u=np.empty((3,) + self.shape),
                       phi=np.empty(self.shape), psi=np.empty(self.shape),
                       C=np.empty(self.shape))
        for k in ("rho", "phi", "psi", "C"):
            a = out[k]
            if a.dtype != np.float64 or a.shape != self.shape or not a.flags.c_contiguous:
                raise ValueError(f"fields: {k} must be a C-contiguous float64 array of {self.shape}")
        a = out["u"]
        if a.dtype != np.float64 or a.shape != (3,) + self.shape or not a.flags.c_contiguous:
            raise ValueError(f"fields: u must be a C-contiguous float64 array of {(3,) + self.shape}")
        self._check(self.L.lbs_get_fields(self.h, *[_dp(out[k]) for k in ("rho", "u", "phi", "psi", "C")]))
        return out

    def profile(self, on=True):
        self._check(self.L.lbs_profile(self.h, int(bool(on))))

    def kernel_times(self):
        """Device milliseconds of each kernel group in the last step."""
        ms = np.zeros(len(KERNEL_GROUPS))
        self._check(self.L.lbs_kernel_times(self.h, _dp(ms), len(KERNEL_GROUPS)))
        return dict(zip(KERNEL_GROUPS, ms.tolist()))

    def set_graph(self, on=True):
        """One CUDA graph per step (default) or individual launches."""
        self._check(self.L.lbs_set_graph(self.h, int(bool(on))))

    def kernel_count(self):
        return int(self.L.lbs_step_kernel_count(self.h))

    def step_result(self):
        """(steps taken, total surfactant before the last rescale, rescale
        factor) after waiting for the queued steps (24 bytes read back)."""
        out = np.empty(3)
        self._check(self.L.lbs_step_result(self.h, _dp(out)))
        return int(out[0]), float(out[1]), float(out[2])

    def save_state(self):
        """Raw copy of the carried state (see lbs_save_state) as bytes."""
        n = C.c_size_t(0)
        self._check(self.L.lbs_save_state(self.h, None, C.byref(n)))
        buf = (C.c_char * n.value)()
        self._check(self.L.lbs_save_state(self.h, buf, C.byref(n)))
        return bytes(buf[:n.value])

    def load_state(self, state):
        """Restore a state written by save_state (see lbs_load_state)."""
        buf = C.create_string_buffer(bytes(state), len(state))
        self._check(self.L.lbs_load_state(self.h, buf, len(state)))

    def set_sor_tile(self, variant):
        """Blocked SOR tile variant of a 2D context (see lbs_set_sor_tile)."""
        self._check(self.L.lbs_set_sor_tile(self.h, int(variant)))

    def set_sor_wait_limit(self, polls):
        """Most polls a block waits at the one-launch SOR's grid barrier
        (see lbs_set_sor_wait_limit)."""
        self._check(self.L.lbs_set_sor_wait_limit(self.h, int(polls)))

    def set_sor_persistent(self, on=True):
        """All SOR rounds of a 2D solve in one launch, or one launch a round
        (see lbs_set_sor_persistent)."""
        self._check(self.L.lbs_set_sor_persistent(self.h, int(bool(on))))

    def macro(self):
        """Intermediate fields of the current state (see lbs_get_macro)."""
        out = dict(g=np.empty((3,) + self.shape), a=np.empty(self.shape),
                   F=np.empty((3,) + self.shape), u=np.empty((3,) + self.shape),
                   S=np.empty(self.shape), B=np.empty(self.shape))
        self._check(self.L.lbs_get_macro(self.h, *[_dp(out[k]) for k in ("g", "a", "F", "u", "S", "B")]))
        return out

    def diagnostics(self):
        d = LbsDiag()
        self._check(self.L.lbs_diagnostics(self.h, C.byref(d)))
        return _diag_dict(d)


def _diag_dict(d):
    return {k: (list(getattr(d, k)) if k in ("U", "centroid") else getattr(d, k))
            for k, _ in LbsDiag._fields_}


class Batch:
    """A batch of independent 2D instances advanced together (lbs_batch_*):
    one launch per phase for all instances, one CUDA graph per 8 steps.
    Workspace: a torch uint8 tensor; work on a torch CUDA stream."""

    def __init__(self, cfgs, storage="f32", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.L = load()
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.n = len(cfgs)
        arr = (LbsParams * self.n)()
        for k, cfg in enumerate(cfgs):
            arr[k] = params_from(cfg, self.storage)
        self.params = arr
        self.shapes = [(1, arr[k].ny, arr[k].nx) for k in range(self.n)]
        nbytes = self.L.lbs_batch_workspace_bytes(arr, self.n, self.storage)
        if nbytes == 0:
            raise LbsError(LBS_EINVAL, "invalid batch parameters")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        r = self.L.lbs_batch_create(arr, self.n, self.storage, C.c_void_p(self.stream.cuda_stream),
                                    C.c_void_p(aligned), nbytes, C.byref(h))
        self.h = h
        self._check(r)

    def _check(self, r):
        if r != LBS_OK:
            msg = self.L.lbs_batch_last_error(self.h).decode() if self.h else "?"
            raise LbsError(r, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.lbs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f(self, k, x, comps=None):
        if x is None:
            return None
        shape = self.shapes[k] if comps is None else (comps,) + self.shapes[k]
        return np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), shape))

    def init_fields(self, k, phi, psi=None, C_=None, u=None):
        arrs = [self._f(k, phi), self._f(k, psi), self._f(k, C_), self._f(k, u, 3)]
        self._check(self.L.lbs_batch_init_fields(self.h, int(k), *[_dp(a) for a in arrs]))

    def set_tiles(self, tx, ty, sor_tile=0):
        self._check(self.L.lbs_batch_set_tiles(self.h, int(tx), int(ty), int(sor_tile)))

    def set_graph(self, on=True):
        self._check(self.L.lbs_batch_set_graph(self.h, int(bool(on))))

    def step(self, n=1):
        self._check(self.L.lbs_batch_step(self.h, int(n)))

    def sync(self):
        self._check(self.L.lbs_batch_sync(self.h))

    def fields(self, k):
        shape = self.shapes[k]
        rho = np.empty(shape)
        u = np.empty((3,) + shape)
        phi, psi, C_ = (np.empty(shape) for _ in range(3))
        self._check(self.L.lbs_batch_get_fields(self.h, int(k), _dp(rho), _dp(u), _dp(phi),
                                                _dp(psi), _dp(C_)))
        return dict(rho=rho, u=u, phi=phi, psi=psi, C=C_)

    def diagnostics(self):
        d = (LbsDiag * self.n)()
        self._check(self.L.lbs_batch_diagnostics(self.h, d))
        return [_diag_dict(d[k]) for k in range(self.n)]

    def kernel_count(self):
        return int(self.L.lbs_batch_step_kernel_count(self.h))

    def status(self):
        """Per-instance status codes since the last call (0 = fine)."""
        st = (C.c_int * self.n)()
        self._check(self.L.lbs_batch_status(self.h, st))
        return list(st)

    def set_active(self, k, on=True):
        self._check(self.L.lbs_batch_set_active(self.h, int(k), int(bool(on))))


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Mlp:
    """Ensemble of fully connected networks trained and evaluated by the
    library's kernels (lbs_mlp_*).  Arrays are float32 numpy, row-major."""

    def __init__(self, members, n_in, width, depth, n_out, max_batch=1024, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.L = load()
        self.E, self.n_in, self.n_out, self.max_batch = members, n_in, n_out, max_batch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        r = self.L.lbs_mlp_create(members, n_in, width, depth, n_out, max_batch,
                                  C.c_void_p(self.stream.cuda_stream), C.byref(h))
        self.h = h
        self._check(r)
        self.P = int(self.L.lbs_mlp_param_count(self.h))

    def _check(self, r):
        if r != LBS_OK:
            msg = self.L.lbs_mlp_last_error(self.h).decode() if self.h else "?"
            raise LbsError(r, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.lbs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _f32(a, shape=None):
        a = np.ascontiguousarray(np.asarray(a, np.float32))
        return a.reshape(shape) if shape is not None else a

    def init(self, seed):
        self._check(self.L.lbs_mlp_init(self.h, C.c_ulonglong(seed)))

    def set_params(self, theta):
        t = self._f32(theta, (self.E * self.P,))
        self._check(self.L.lbs_mlp_set_params(self.h, _fp(t)))

    def params(self):
        out = np.empty(self.E * self.P, np.float32)
        self._check(self.L.lbs_mlp_get_params(self.h, _fp(out)))
        return out.reshape(self.E, self.P)

    def forward(self, x, bf16=False):
        """x [E][B][n_in] -> y [E][B][n_out]."""
        x = self._f32(x)
        B = x.shape[1]
        y = np.empty((self.E, B, self.n_out), np.float32)
        self._check(self.L.lbs_mlp_forward(self.h, _fp(x), B, int(bool(bf16)), _fp(y)))
        return y

    def gradient(self, x, t):
        """(loss [E], grad [E][P]) for x [E][B][n_in], t [E][B][n_out]."""
        x, t = self._f32(x), self._f32(t)
        g = np.empty(self.E * self.P, np.float32)
        loss = np.empty(self.E)
        self._check(self.L.lbs_mlp_gradient(self.h, _fp(x), _fp(t), x.shape[1], _fp(g), _dp(loss)))
        return loss, g.reshape(self.E, self.P)

    def set_grad(self, g):
        g = self._f32(g, (self.E * self.P,))
        self._check(self.L.lbs_mlp_set_grad(self.h, _fp(g)))

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.L.lbs_mlp_adam_step(self.h, lr, beta1, beta2, eps))

    def set_data(self, X, Y):
        X, Y = self._f32(X), self._f32(Y)
        self._check(self.L.lbs_mlp_set_data(self.h, _fp(X), _fp(Y), X.shape[0]))

    def train(self, iters, batch, lr, seed, beta1=0.9, beta2=0.999, eps=1e-8):
        loss = np.empty(self.E)
        self._check(self.L.lbs_mlp_train(self.h, int(iters), int(batch), lr, beta1, beta2, eps,
                                         C.c_ulonglong(seed), _dp(loss)))
        return loss

    def predict(self, x, bf16=True):
        """Ensemble mean and standard deviation [n][n_out] for x [n][n_in]."""
        x = self._f32(x)
        n = x.shape[0]
        mean = np.empty((n, self.n_out), np.float32)
        sd = np.empty((n, self.n_out), np.float32)
        self._check(self.L.lbs_mlp_predict(self.h, _fp(x), n, int(bool(bf16)), _fp(mean), _fp(sd)))
        return mean, sd
