"""The C-ABI library builds, loads and exports every entry point that
include/lbs.h declares (no GPU needed: nothing is called that computes)."""
import ctypes
import os
import re

import pytest

import paper_2311_15242_gb300 as P
from paper_2311_15242_gb300 import lbs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "lbs.h")).read()
    pat = r"^(?:int|void|size_t|const char)\s*\*?\s*(lbs_[a-z_0-9]+)\s*\("
    return sorted(set(re.findall(pat, txt, flags=re.M)))


def test_header_and_binding_agree():
    assert declared() == sorted(lbs.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = P.load()
    for name in declared():
        assert hasattr(L, name), name


def test_param_struct_layout_matches_header():
    """ctypes mirror of lbs_params: size equals the C struct (sizeof via the
    defaults call writing every field) and defaults are the paper's values."""
    p = lbs.LbsParams()
    assert P.load().lbs_params_default(ctypes.byref(p), 64, 32, 1) == 0
    assert (p.nx, p.ny, p.nz) == (64, 32, 1)
    assert p.beta == 0.7 and p.sor_omega == 1.2 and p.sigma_min_ratio == 0.1
    assert abs(p.alphaR - 4 / 9) < 1e-15


def test_workspace_and_validation_on_host():
    L = P.load()
    p = lbs.LbsParams()
    L.lbs_params_default(ctypes.byref(p), 64, 32, 1)
    assert L.lbs_workspace_bytes(ctypes.byref(p), lbs.LBS_F32) > 0
    assert L.lbs_workspace_bytes(ctypes.byref(p), lbs.LBS_F64) > L.lbs_workspace_bytes(ctypes.byref(p), lbs.LBS_F32)
    bad = lbs.LbsParams()
    L.lbs_params_default(ctypes.byref(bad), 64, 32, 1)
    bad.rhoR0 = -1.0
    assert L.lbs_workspace_bytes(ctypes.byref(bad), lbs.LBS_F32) == 0
    bad.rhoR0 = 1.0
    bad.wall[0] = 1
    bad.nx = 2
    assert L.lbs_workspace_bytes(ctypes.byref(bad), lbs.LBS_F32) == 0
    h = ctypes.c_void_p()
    assert L.lbs_create(ctypes.byref(bad), lbs.LBS_F32, None, None, 0, ctypes.byref(h)) == lbs.LBS_EINVAL
    assert b"3 nodes" in L.lbs_last_error(h)
    L.lbs_destroy(h)
    # mirror planes (2) are accepted; other axis codes and moving mirrors not
    ok = lbs.LbsParams()
    L.lbs_params_default(ctypes.byref(ok), 63, 31, 1)
    ok.wall[0] = ok.wall[1] = 2
    assert L.lbs_workspace_bytes(ctypes.byref(ok), lbs.LBS_F32) > 0
    ok.wall[1] = 3
    assert L.lbs_workspace_bytes(ctypes.byref(ok), lbs.LBS_F32) == 0
    ok.wall[1] = 2
    ok.uw_lo[1][0] = 0.01
    assert L.lbs_workspace_bytes(ctypes.byref(ok), lbs.LBS_F32) == 0


def test_3d_validation_on_host():
    """D3Q19 grids: accepted with even periodic axes (any size on a walled
    axis), refused with an odd periodic axis (the in-place red-black SOR
    would couple cells of one colour across the seam); a 2D grid cannot
    have walls on z.  The 3D workspace holds 19 population planes per set."""
    L = P.load()
    p = lbs.LbsParams()
    L.lbs_params_default(ctypes.byref(p), 34, 20, 17)
    p.wall[2] = 1
    b3 = L.lbs_workspace_bytes(ctypes.byref(p), lbs.LBS_F32)
    assert b3 > 0
    assert abs(p.alphaR - 1 / 3) < 1e-15
    p.nx = 33
    assert L.lbs_workspace_bytes(ctypes.byref(p), lbs.LBS_F32) == 0
    h = ctypes.c_void_p()
    assert L.lbs_create(ctypes.byref(p), lbs.LBS_F32, None, None, 0, ctypes.byref(h)) == lbs.LBS_EINVAL
    assert b"even size on periodic axis 0" in L.lbs_last_error(h)
    L.lbs_destroy(h)
    p.wall[0] = 1  # odd is fine on a walled axis
    assert L.lbs_workspace_bytes(ctypes.byref(p), lbs.LBS_F32) > 0
    q = lbs.LbsParams()
    L.lbs_params_default(ctypes.byref(q), 34, 20, 1)
    q.wall[2] = 1
    assert L.lbs_workspace_bytes(ctypes.byref(q), lbs.LBS_F32) == 0
    # populations: 4 sets x 19 planes (3D) against 4 x 9 (2D) of the same cells
    q.wall[2] = 0
    q.ny = 20 * 17
    b2 = L.lbs_workspace_bytes(ctypes.byref(q), lbs.LBS_F32)
    assert b3 > b2


def test_no_cpu_fallback_without_a_device():
    """Without a CUDA device every entry point of the binding refuses to run
    (no CPU fallback); the check is skipped where a device exists."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import workloads as W
    from paper_2311_15242_gb300 import Batch, Mlp, Solver
    with pytest.raises(RuntimeError, match="CUDA device"):
        Solver(W.droplet_adsorption_2d(n=16, R=4.0))
    with pytest.raises(RuntimeError, match="CUDA device"):
        Batch([W.droplet_adsorption_2d(n=16, R=4.0)])
    with pytest.raises(RuntimeError, match="CUDA device"):
        Mlp(1, 5, 8, 1, 2)
