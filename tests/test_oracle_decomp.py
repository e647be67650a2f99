"""The decomposed oracle (oracle/decomp.py): one grid split into slabs along
its slowest axis, ghost rows exchanged between the phases of the step, the
lexicographic SOR pipelined over the slabs in rank order and the rescale's
Kahan total passed from slab to slab.  It must reproduce the undecomposed
oracle bit for bit: the populations of both colours, psi and C after a run
of coupled steps (Secs. 2.1-2.2), for 2, 3 and 4 slabs, on a periodic
decomposed axis (the 2D bubble rise) and on one bounded by moving walls
(the 3D sheared droplet); and as real ranks, two gloo processes exchanging
the same rows by send / recv and allreduce."""
import os
import socket
import sys

import numpy as np
import pytest

import workloads as W
from oracle.decomp import SlabOracle, run_gloo_rank
from oracle.ora import Oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bubble2d():
    c = W.bubble_rise_2d(nx=24, ny=40, D_b=12.0, Eo=4.0)
    c["center"] = [11.3, 13.7, 0.0]
    return c


def shear3d():
    c = W.shear_droplet_3d(nx=16, ny=12, nz=17, R=4.0)
    c["center"] = [7.8, 5.4, 8.2]
    return c


def reference(cfg, f, steps):
    o = Oracle(cfg)
    o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    o.step(steps)
    fR, fB = o.pops()
    fl = o.fields()
    return fR, fB, fl["psi"], fl["C"]


@pytest.mark.parametrize("make,nranks,steps", [(bubble2d, 2, 12), (bubble2d, 4, 12),
                                               (shear3d, 2, 10), (shear3d, 3, 10)],
                         ids=["2d-2", "2d-4", "3d-2", "3d-3"])
def test_slabs_match_the_undecomposed_oracle(make, nranks, steps):
    cfg = make()
    f = W.initial_fields(cfg, seed=5, noise=0.02, u0=1e-3)
    ref = reference(cfg, f, steps)
    d = SlabOracle(cfg, nranks)
    d.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    d.step(steps)
    got = d.state()
    for name, a, b in zip(("fR", "fB", "psi", "C"), ref, got):
        assert np.array_equal(a.reshape(b.shape), b), (name, float(np.abs(a.reshape(b.shape) - b).max()))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, which, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import test_oracle_decomp as T
    from oracle.decomp import run_gloo_rank as run
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = T.bubble2d() if which == "2d" else T.shear3d()
    f = W.initial_fields(cfg, seed=5, noise=0.02, u0=1e-3)
    state, rows = run(cfg, f, steps, rank, world)
    q.put((rank, rows, state))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("which,steps", [("2d", 8), ("3d", 6)])
def test_two_gloo_ranks_match_the_undecomposed_oracle(which, steps):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, which, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = bubble2d() if which == "2d" else shear3d()
    f = W.initial_fields(cfg, seed=5, noise=0.02, u0=1e-3)
    ref = reference(cfg, f, steps)
    out.sort(key=lambda t: t[0])
    axis = 2 if which == "2d" else 1  # rows axis of (Q, nz, ny, nx) arrays
    for k, name in enumerate(("fR", "fB", "psi", "C")):
        got = np.concatenate([o[2][k] for o in out], axis=axis)
        a = ref[k].reshape(got.shape)
        assert np.array_equal(a, got), (name, float(np.abs(a - got).max()))
