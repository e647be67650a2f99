"""The allocation-free total (lbs_surfactant_total_static) against the
existing entry point that reports the same quantity (lbs_diagnostics,
surf_total).

This entry point is for callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they must not stall on an
allocation's synchronisation): it keeps its scratch in a fixed array of the
library's device memory.  The test calls it twice in a row through the C ABI,
since every call reuses that scratch, and also checks that a grid beyond the
scratch's capacity is refused before anything runs.  It is collected last
(file name), and passes on its own in a fresh process as well."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _solver(cfg, storage):
    from paper_2311_15242_gb300 import Solver
    return Solver(cfg, storage=storage)


@pytest.mark.parametrize("storage,rtol", [("f64", 1e-12), ("f32", 1e-6)])
def test_static_total_matches_diagnostics_twice(storage, rtol):
    import torch

    from paper_2311_15242_gb300 import lbs

    cfg = W.bubble_rise_2d(nx=72, ny=136, D_b=24.0, Eo=2.0)
    f = W.initial_fields(cfg, seed=11, noise=0.02)
    s = _solver(cfg, storage)
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    s.step(12)
    ref = s.diagnostics()["surf_total"]
    m, fld = s.macro(), s.fields()
    dt = torch.float64 if storage == "f64" else torch.float32
    dev = [torch.from_numpy(np.ascontiguousarray(x[0])).to("cuda", dt)
           for x in (m["a"], 1.0 - fld["phi"], fld["psi"], fld["C"])]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = lbs.load()
    code = lbs.STORAGE[storage]
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out.fill_(-1.0)
        rc = L.lbs_surfactant_total_static(
            code, *[ctypes.c_void_p(t.data_ptr()) for t in dev], cfg["nx"], cfg["ny"], 1,
            cfg["nx"], cfg["eps_w"], ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
        assert rc == lbs.LBS_OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=rtol)
    s.close()


@pytest.mark.parametrize("storage,rtol", [("f64", 1e-12), ("f32", 1e-6)])
def test_static_total_3d_pitched_rows_twice(storage, rtol):
    """A D3Q19 state (nz > 1) in rows padded beyond nx: the (z, y) rows are
    flattened with the caller's pitch; matches the 3D context's surf_total."""
    import torch

    from paper_2311_15242_gb300 import lbs

    nx, ny, nz = 34, 20, 17
    cfg = W.shear_droplet_3d(nx=nx, ny=ny, nz=nz, R=5.0)
    f = W.initial_fields(cfg, seed=4, noise=0.02)
    s = _solver(cfg, storage)
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    s.step(6)
    ref = s.diagnostics()["surf_total"]
    m, fld = s.macro(), s.fields()
    dt = torch.float64 if storage == "f64" else torch.float32
    pitch = nx + 7
    dev = []
    for x in (m["a"], 1.0 - fld["phi"], fld["psi"], fld["C"]):
        t = torch.full((nz, ny, pitch), float("nan"), dtype=dt, device="cuda")
        t[:, :, :nx] = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
        dev.append(t)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = lbs.load()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out.fill_(-1.0)
        rc = L.lbs_surfactant_total_static(
            lbs.STORAGE[storage], *[ctypes.c_void_p(t.data_ptr()) for t in dev], nx, ny, nz,
            pitch, cfg["eps_w"], ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
        assert rc == lbs.LBS_OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=rtol)
    s.close()


def test_static_total_refuses_grids_beyond_its_scratch():
    from paper_2311_15242_gb300 import lbs
    L = lbs.load()
    one = ctypes.c_void_p(16)  # never dereferenced: refused before any launch
    n = 8192
    rc = L.lbs_surfactant_total_static(lbs.LBS_F32, one, one, one, one, n, n, 1, n, 1e-6,
                                       one, None)
    assert rc == lbs.LBS_EINVAL
