"""The oracle on a grid decomposed into slabs: the domain-decomposition
reference for a multi-GPU step (one large grid split along its slowest
axis, one slab per rank).

Test infrastructure only.  Each slab is an oracle context of its own rows
plus G ghost rows on every side where it meets another slab (none at a wall
of the axis); the phases of the coupled step (Secs. 2.1-2.2) run per slab,
and between them the ghost rows are refreshed from the neighbours:

  - before the lattice Boltzmann part (fields at t, explicit terms,
    collision, recolouring, streaming): populations, psi and C.  Their
    stencils chain to a depth of 4 rows (colour gradient -> normals ->
    curvature -> velocity -> WENO3 terms; velocity -> correction term ->
    collision -> streaming), within G = 5;
  - before the fields at t+1 (the weights of the Crank-Nicolson solve):
    the streamed populations;
  - in the SOR: the rows next to the slab before each slab's sweep.  The
    oracle's SOR is lexicographic (x fastest, then y, then z); with slabs
    along the slowest axis the slabs sweep one after another in rank order,
    each seeing its lower neighbour's rows of the current sweep and its
    upper neighbour's rows of the previous one, exactly as the undecomposed
    sweep does.  The stop test uses the maxima over all slabs (an
    allreduce of two numbers);
  - the total surfactant of the rescale: the Kahan sum is passed from slab
    to slab in rank order (an exclusive scan of the compensated sum), so it
    adds the cells in the undecomposed order.

The results are therefore those of the undecomposed oracle bit for bit;
tests/test_oracle_decomp.py checks it for 2 and 4 slabs.  SlabOracle holds
every slab in one process (emulated ranks); run_gloo_rank runs one slab per
process and exchanges the same rows over torch.distributed (gloo).
"""
import ctypes as C

import numpy as np

from .ora import Oracle, lib

GHOST = 5


def split_rows(n, nranks):
    """Contiguous row ranges [r0, r1) of nearly equal size."""
    base, extra = divmod(n, nranks)
    out, r0 = [], 0
    for r in range(nranks):
        r1 = r0 + base + (1 if r < extra else 0)
        out.append((r0, r1))
        r0 = r1
    return out


class Slab:
    """One slab: owned rows [r0, r1) of the global axis, lo / hi ghost rows."""

    def __init__(self, cfg, axis, r0, r1, glo, ghi, end_lo, end_hi):
        self.r0, self.r1, self.glo, self.ghi = r0, r1, glo, ghi
        self.owned = r1 - r0
        self.nloc = self.owned + glo + ghi
        local = dict(cfg)
        local["ny" if axis == 1 else "nz"] = self.nloc
        self.o = Oracle(local)
        lib().ora_set_ends(self.o.h, axis, end_lo, end_hi)
        self.axis = axis
        self.D = self.o.D
        self.Q = self.o.Q

    def field(self, name):
        """numpy view of an array of the slab's context: ([Q], nz, ny, nx)."""
        q = self.Q if name in ("fR", "fB") else 1
        shape = (q,) + self.o.shape
        ptr = lib().ora_field(self.o.h, name.encode())
        return np.ctypeslib.as_array(ptr, shape=shape)

    def rows(self, arr, k0, k1):
        """arr[..., local rows k0:k1 of the decomposed axis]."""
        return arr[:, :, k0:k1, :] if self.axis == 1 else arr[:, k0:k1, :, :]


class SlabOracle:
    """The oracle on cfg's grid split into `nranks` slabs (emulated ranks in
    one process), stepping exactly like Oracle(cfg)."""

    def __init__(self, cfg, nranks, ghost=GHOST):
        self.cfg = cfg
        D = 2 if cfg.get("nz", 1) == 1 else 3
        self.axis = 1 if D == 2 else 2
        self.n = cfg["ny"] if D == 2 else cfg["nz"]
        self.wall = cfg["wall"][self.axis]
        self.periodic = self.wall == 0
        self.slabs = []
        ranges = split_rows(self.n, nranks)
        for r, (r0, r1) in enumerate(ranges):
            at_lo = r == 0 and not self.periodic
            at_hi = r == nranks - 1 and not self.periodic
            self.slabs.append(Slab(cfg, self.axis, r0, r1, 0 if at_lo else ghost,
                                   0 if at_hi else ghost, self.wall if at_lo else 0,
                                   self.wall if at_hi else 0))
        self.M0 = None

    # ---- ghost exchange -------------------------------------------------
    def _global_rows(self, name):
        """The global array of `name` assembled from the slabs' owned rows."""
        parts = [s.rows(s.field(name), s.glo, s.glo + s.owned) for s in self.slabs]
        return np.concatenate(parts, axis=2 if self.axis == 1 else 1)

    def _fill(self, s, name, glob):
        """Every row of slab s from the global array (ghost rows wrap on a
        periodic axis; slabs at a wall have no ghost rows there)."""
        arr = s.field(name)
        src = (np.arange(s.nloc) + s.r0 - s.glo) % self.n
        if self.axis == 1:
            arr[:, :, :, :] = glob[:, :, src, :]
        else:
            arr[:, :, :, :] = glob[:, src, :, :]

    def exchange(self, names, only=None):
        for name in names:
            glob = self._global_rows(name)
            for k, s in enumerate(self.slabs):
                if only is None or k == only:
                    self._fill(s, name, glob)

    # ---- state ------------------------------------------------------------
    def init_fields(self, phi, psi, C_, u=None):
        ax = self.axis
        for s in self.slabs:
            src = (np.arange(s.nloc) + s.r0 - s.glo) % self.n
            take = (lambda a: a[:, src, :]) if ax == 1 else (lambda a: a[src, :, :])
            takev = (lambda a: a[:, :, src, :]) if ax == 1 else (lambda a: a[:, src, :, :])
            s.o.init_fields(take(np.asarray(phi)), take(np.asarray(psi)), take(np.asarray(C_)),
                            None if u is None else takev(np.asarray(u)))
        self.M0 = self._total()
        for s in self.slabs:
            lib().ora_set_M0(s.o.h, self.M0)

    def _total(self):
        ks = (C.c_double * 2)(0.0, 0.0)
        for s in self.slabs:
            lib().ora_surf_rows(s.o.h, s.glo, s.glo + s.owned, ks)
        return ks[0]

    def state(self):
        """(fR, fB, psi, C) of the whole grid, from the owned rows."""
        return tuple(self._global_rows(n) for n in ("fR", "fB", "psi", "C"))

    # ---- one step ----------------------------------------------------------
    def step(self, n=1):
        for _ in range(n):
            self._step()

    def _step(self):
        L = lib()
        p = self.cfg
        self.exchange(["fR", "fB", "psi", "C"])
        for s in self.slabs:
            L.ora_phase(s.o.h, 0)
        if not p.get("transport", 1):
            for s in self.slabs:
                L.ora_finish(s.o.h, 1.0, 0.0, 0, 0)
            return
        for s in self.slabs:
            L.ora_phase(s.o.h, 1)
        self.exchange(["fR", "fB"])
        for s in self.slabs:
            L.ora_phase(s.o.h, 2)
        its = []
        tol = float(s.o.p.sor_tol)
        max_it = int(s.o.p.sor_max_iter)
        for which, wphase, name in ((0, 3, "psi"), (1, 4, "C")):
            for s in self.slabs:
                L.ora_phase(s.o.h, wphase)
            it_used = -1
            for it in range(1, max_it + 1):
                md, mx = C.c_double(0.0), C.c_double(0.0)
                for k, s in enumerate(self.slabs):
                    self.exchange([name], only=k)
                    L.ora_sor_rows(s.o.h, which, s.glo, s.glo + s.owned, C.byref(md), C.byref(mx))
                if md.value <= tol * mx.value:
                    it_used = it
                    break
            its.append(it_used)
        if its[0] < 0 or its[1] < 0:
            raise RuntimeError("oracle SOR did not converge")
        Mt = self._total()
        scale = self.M0 / Mt if Mt > 0 else 1.0
        for s in self.slabs:
            L.ora_finish(s.o.h, scale, Mt, its[0], its[1])


def run_gloo_rank(cfg, fields, steps, rank, world, ghost=GHOST):
    """One slab of a decomposed oracle in this process (rank `rank` of
    `world`, torch.distributed already initialised with gloo).  Ghost rows
    travel by send / recv, the SOR stop test and the total by allreduce /
    a scan over the ranks.  Returns the slab's (fR, fB, psi, C) owned rows
    and its row range."""
    import torch
    import torch.distributed as dist

    grid = SlabOracle.__new__(SlabOracle)
    grid.cfg = cfg
    D = 2 if cfg.get("nz", 1) == 1 else 3
    grid.axis = 1 if D == 2 else 2
    grid.n = cfg["ny"] if D == 2 else cfg["nz"]
    grid.wall = cfg["wall"][grid.axis]
    grid.periodic = grid.wall == 0
    r0, r1 = split_rows(grid.n, world)[rank]
    at_lo = rank == 0 and not grid.periodic
    at_hi = rank == world - 1 and not grid.periodic
    s = Slab(cfg, grid.axis, r0, r1, 0 if at_lo else ghost, 0 if at_hi else ghost,
             grid.wall if at_lo else 0, grid.wall if at_hi else 0)
    lo_nb = (rank - 1) % world if not at_lo else None
    hi_nb = (rank + 1) % world if not at_hi else None
    L = lib()

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a))

    def send_recv(name, lo_rows, hi_rows):
        """Send this slab's edge rows to the neighbours and receive their
        edge rows into this slab's ghost rows (lo_rows / hi_rows deep)."""
        arr = s.field(name)
        reqs, bufs = [], []
        if lo_nb is not None and lo_rows:
            reqs.append(dist.isend(t(s.rows(arr, s.glo, s.glo + lo_rows)).clone(), lo_nb, tag=1))
        if hi_nb is not None and hi_rows:
            reqs.append(dist.isend(
                t(s.rows(arr, s.glo + s.owned - hi_rows, s.glo + s.owned)).clone(), hi_nb, tag=2))
        if hi_nb is not None and hi_rows:
            b = t(s.rows(arr, s.glo + s.owned, s.glo + s.owned + hi_rows)).clone()
            dist.recv(b, hi_nb, tag=1)
            bufs.append((s.glo + s.owned, b))
        if lo_nb is not None and lo_rows:
            b = t(s.rows(arr, s.glo - lo_rows, s.glo)).clone()
            dist.recv(b, lo_nb, tag=2)
            bufs.append((s.glo - lo_rows, b))
        for q in reqs:
            q.wait()
        for k0, b in bufs:
            v = s.rows(arr, k0, k0 + b.shape[2 if grid.axis == 1 else 1])
            v[...] = b.numpy()

    # initial state of the slab's rows (ghosts included) and the global M0
    src = (np.arange(s.nloc) + s.r0 - s.glo) % grid.n
    ax = grid.axis
    take = (lambda a: a[:, src, :]) if ax == 1 else (lambda a: a[src, :, :])
    takev = (lambda a: a[:, :, src, :]) if ax == 1 else (lambda a: a[:, src, :, :])
    s.o.init_fields(take(fields["phi"]), take(fields["psi"]), take(fields["C"]),
                    None if fields.get("u") is None else takev(fields["u"]))

    def chained_total():
        ks = (C.c_double * 2)(0.0, 0.0)
        if rank > 0:
            b = torch.zeros(2, dtype=torch.float64)
            dist.recv(b, rank - 1, tag=3)
            ks[0], ks[1] = float(b[0]), float(b[1])
        L.ora_surf_rows(s.o.h, s.glo, s.glo + s.owned, ks)
        if rank < world - 1:
            dist.send(torch.tensor([ks[0], ks[1]], dtype=torch.float64), rank + 1, tag=3)
        tot = torch.tensor([ks[0] if rank == world - 1 else 0.0], dtype=torch.float64)
        dist.broadcast(tot, world - 1)
        return float(tot[0])

    M0 = chained_total()
    L.ora_set_M0(s.o.h, M0)
    tol = float(s.o.p.sor_tol)
    max_it = int(s.o.p.sor_max_iter)
    for _ in range(steps):
        for name in ("fR", "fB", "psi", "C"):
            send_recv(name, s.glo, s.ghi)
        L.ora_phase(s.o.h, 0)
        if not cfg.get("transport", 1):
            L.ora_finish(s.o.h, 1.0, 0.0, 0, 0)
            continue
        L.ora_phase(s.o.h, 1)
        for name in ("fR", "fB"):
            send_recv(name, s.glo, s.ghi)
        L.ora_phase(s.o.h, 2)
        its = []
        for which, wphase, name in ((0, 3, "psi"), (1, 4, "C")):
            L.ora_phase(s.o.h, wphase)
            it_used = -1
            arr = s.field(name)
            lo_g = (s.glo - 1, s.glo)                      # lower ghost row
            hi_g = (s.glo + s.owned, s.glo + s.owned + 1)  # upper ghost row
            first = (s.glo, s.glo + 1)
            last = (s.glo + s.owned - 1, s.glo + s.owned)
            wrap = grid.periodic and world > 1
            for it in range(1, max_it + 1):
                reqs = []
                # rows of the previous sweep: every rank's first row to its
                # lower neighbour (its upper ghost); on a periodic axis the
                # last rank's last row to rank 0 (its lower ghost)
                if rank > 0:
                    reqs.append(dist.isend(t(s.rows(arr, *first)).clone(), rank - 1, tag=11))
                if wrap and rank == world - 1:
                    reqs.append(dist.isend(t(s.rows(arr, *last)).clone(), 0, tag=12))
                if rank < world - 1:
                    b = t(s.rows(arr, *hi_g)).clone()
                    dist.recv(b, rank + 1, tag=11)
                    s.rows(arr, *hi_g)[...] = b.numpy()
                if wrap and rank == 0:
                    b = t(s.rows(arr, *lo_g)).clone()
                    dist.recv(b, world - 1, tag=12)
                    s.rows(arr, *lo_g)[...] = b.numpy()
                # rows of this sweep: the lower neighbour's last row; on a
                # periodic axis the last rank also waits for rank 0's first
                if rank > 0:
                    b = t(s.rows(arr, *lo_g)).clone()
                    dist.recv(b, rank - 1, tag=13)
                    s.rows(arr, *lo_g)[...] = b.numpy()
                if wrap and rank == world - 1:
                    b = t(s.rows(arr, *hi_g)).clone()
                    dist.recv(b, 0, tag=14)
                    s.rows(arr, *hi_g)[...] = b.numpy()
                md, mx = C.c_double(0.0), C.c_double(0.0)
                L.ora_sor_rows(s.o.h, which, s.glo, s.glo + s.owned, C.byref(md), C.byref(mx))
                if rank < world - 1:
                    reqs.append(dist.isend(t(s.rows(arr, *last)).clone(), rank + 1, tag=13))
                if wrap and rank == 0:
                    reqs.append(dist.isend(t(s.rows(arr, *first)).clone(), world - 1, tag=14))
                for q in reqs:
                    q.wait()
                m = torch.tensor([md.value, mx.value], dtype=torch.float64)
                dist.all_reduce(m, op=dist.ReduceOp.MAX)
                if float(m[0]) <= tol * float(m[1]):
                    it_used = it
                    break
            its.append(it_used)
        Mt = chained_total()
        L.ora_finish(s.o.h, M0 / Mt if Mt > 0 else 1.0, Mt, its[0], its[1])
    return tuple(s.rows(s.field(n), s.glo, s.glo + s.owned).copy()
                 for n in ("fR", "fB", "psi", "C")), (r0, r1)
