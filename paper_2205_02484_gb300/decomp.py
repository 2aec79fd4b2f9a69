"""Phi-slab decomposition of the step: the slab layout of the paper's
multi-GPU runs (Section 3), split along phi, over contexts whose X3 ghosts
are external (BC_EXTERNAL).

One step of the decomposed grid:
  1. every slab runs the predictor (Eq. 25) and reports its per-direction
     CFL minima (the terms of Eq. 27);
  2. the NG = 3 X3 ghost planes of P-hat are exchanged with the phi
     neighbours (periodic in phi);
  3. every slab runs the corrector (Eq. 26);
  4. the ghost planes of P are exchanged;
  5. the minima are reduced over slabs by a minimum, and every slab advances
     t and sets the next dt from Eq. 27.
The metric does not depend on phi, each slab's ghost planes hold exactly the
values the undecomposed grid would read there (taken after the neighbour's
own X1/X2 boundary fill), and a minimum is exact, so the decomposed step
equals the undecomposed one bit for bit -- provided a slab's dX3 equals the
whole grid's, which slab_grid guarantees for power-of-two slab widths.

Two drivers, both over any object with the SlabEngine methods:
  SlabRing -- all slabs on one device and one stream; the exchange is a pack
              and an unpack through device buffers;
  SlabRank -- one slab per process; the exchange is point-to-point sends of
              torch.distributed, the dt reduction a MIN all-reduce.
CtxSlab is the engine over the CUDA library.
"""
from __future__ import annotations

import contextlib
import math

import torch

from . import grmhd as G

NG = G.NG


def slab_grid(base: G.GridParams, R: int) -> G.GridParams:
    """Grid parameters of one of R phi slabs of `base` (n3 / R zones, X3
    ghosts external).  The step uses a slab's phi position nowhere (the
    metric is axisymmetric, the Minkowski box uniform), only dX3, so every
    slab spans [0, (n3 / R) dX3)."""
    if R < 1 or base.n3 % R:
        raise ValueError(f"n3 = {base.n3} does not split into {R} slabs")
    n3 = base.n3 // R
    if n3 < NG:
        raise ValueError(f"slabs of {n3} < {NG} phi zones")
    h = 2.0 * math.pi / base.n3 if base.metric == G.KERR_MKS else (base.x3max - base.x3min) / base.n3
    g = G.GridParams.from_buffer_copy(base)
    g.n3, g.bc3, g.x3min, g.x3max = n3, G.BC_EXTERNAL, 0.0, n3 * h
    return g


def split_phi(x, R: int, r: int):
    """Slab r's part of a (fields, n1, n2, n3) array (numpy or torch), contiguous."""
    n3 = x.shape[3] // R
    part = x[..., r * n3:(r + 1) * n3]
    return part.contiguous() if isinstance(x, torch.Tensor) else part.copy(order="C")


class CtxSlab:
    """SlabEngine over one grmhd context with bc3 = BC_EXTERNAL.  Every call
    is asynchronous on the context's stream (`stream`)."""

    def __init__(self, ctx: G.Context, stream: torch.cuda.Stream):
        if ctx.grid.bc3 != G.BC_EXTERNAL:
            raise ValueError("a slab context needs bc3 = BC_EXTERNAL")
        self.ctx = ctx
        self.stream = stream
        self.device = torch.device("cuda", ctx.grid.device)
        self.dtype = torch.float64 if ctx.grid.precision == G.FP64 else torch.float32
        self.plane_numel = G.x3_plane_bytes(ctx) // (8 if self.dtype == torch.float64 else 4)

    @classmethod
    def create(cls, grid: G.GridParams, phys: G.PhysParams, a: float, stream: torch.cuda.Stream):
        g = G.GridParams.from_buffer_copy(grid)
        g.stream = stream.cuda_stream
        ctx = G.init_grid(g, phys)
        G.set_metric(ctx, a, g.metric)
        return cls(ctx, stream)

    def set_state(self, P, U, t, dt):
        G.set_state(self.ctx, P, U, t, dt)

    def get_state(self):
        return G.get_state(self.ctx)

    def diagnostics(self):
        return G.diagnostics(self.ctx)

    def diag_partials(self, r_bar_max):
        out = torch.empty(G.DIAG_NPART, dtype=torch.float64, device=self.device)
        G.diag_partials(self.ctx, r_bar_max, out)  # on the context stream
        return out

    def diag_combine(self, parts):
        return G.diag_combine(self.ctx, parts)

    def stage(self, st):
        G.stage(self.ctx, st)

    def dtd(self, out, accumulate=False):
        G.step_dtd(self.ctx, out, accumulate)

    def finish(self, dtd):
        G.finish_step(self.ctx, dtd)

    def pack(self, which, side, buf):
        G.x3_pack(self.ctx, which, side, buf)

    def unpack(self, which, side, buf):
        G.x3_unpack(self.ctx, which, side, buf)

    def close(self):
        self.ctx.close()


def _combine(engine, parts):
    """Whole-grid diagnostics from the slabs' partial vectors (one row per
    slab, in slab order), combined by the library on the device (integrals
    and counters summed in that order, div B the largest, Eq. 42, the
    efficiency and the Eq. 43 quotient formed there): (dict, barycentric)."""
    with _stream_of(engine):
        stacked = torch.stack(parts).contiguous()
    return engine.diag_combine(stacked)


def _stream_of(engine):
    s = getattr(engine, "stream", None)
    return torch.cuda.stream(s) if s is not None else contextlib.nullcontext()


class SlabRing:
    """All slabs of one grid on one device, in phi order, sharing one stream.
    A step of library slabs is a fixed sequence of device work on that stream
    (no host read in it), so it is captured once into a CUDA graph and
    replayed.  The graph holds every context's grid record by value: after a
    call that changes one (set_metric, set_learned_guess) call drop_graph().
    set_state writes into the buffers the graph reads and needs nothing."""

    def __init__(self, engines):
        self.e = list(engines)
        e0 = self.e[0]
        self.lo = [torch.empty(e.plane_numel, dtype=e.dtype, device=e.device) for e in self.e]
        self.hi = [torch.empty(e.plane_numel, dtype=e.dtype, device=e.device) for e in self.e]
        self.dtd_buf = torch.empty(3, dtype=torch.float64, device=e0.device)
        self._graph = None
        streams = {id(getattr(e, "stream", None)) for e in self.e}
        self._capturable = all(isinstance(e, CtxSlab) for e in self.e) and len(streams) == 1

    @classmethod
    def create(cls, grid: G.GridParams, phys: G.PhysParams, R: int, a: float, stream=None):
        stream = stream or torch.cuda.Stream(device=grid.device)
        sg = slab_grid(grid, R)
        return cls([CtxSlab.create(sg, phys, a, stream) for _ in range(R)])

    def set_state(self, P, U, t, dt):
        """P, U: the whole grid's state (host arrays or device tensors)."""
        R = len(self.e)
        for r, e in enumerate(self.e):
            with _stream_of(e):  # a device slice is copied on the slab's stream
                e.set_state(split_phi(P, R, r), split_phi(U, R, r), t, dt)
        self.exchange(0)

    def exchange(self, which):
        R = len(self.e)
        for r, e in enumerate(self.e):
            e.pack(which, 0, self.lo[r])
            e.pack(which, 1, self.hi[r])
        for r, e in enumerate(self.e):
            e.unpack(which, 0, self.hi[(r - 1) % R])
            e.unpack(which, 1, self.lo[(r + 1) % R])

    def _step_once(self):
        for r, e in enumerate(self.e):
            e.stage(0)
            e.dtd(self.dtd_buf, accumulate=r > 0)
        self.exchange(1)
        for e in self.e:
            e.stage(1)
        self.exchange(0)
        for e in self.e:
            e.finish(self.dtd_buf)

    def step(self, nsteps=1, graph=True):
        """nsteps RK2 steps of the whole grid; graph=False launches every
        kernel from the host (the form the engines' tests drive)."""
        if not (graph and self._capturable):
            for _ in range(nsteps):
                self._step_once()
            return
        s = self.e[0].stream
        if self._graph is None:
            self._graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self._graph, stream=s):
                self._step_once()
        with torch.cuda.stream(s):
            for _ in range(nsteps):
                self._graph.replay()

    def drop_graph(self):
        self._graph = None

    def diagnostics(self, r_bar_max=80.0):
        return _combine(self.e[0], [e.diag_partials(r_bar_max) for e in self.e])[0]

    def barycentric_radius(self, r_bar_max=80.0):
        """(<r>, mass, numerator) of Eq. 43 over the whole grid: the slabs'
        sums added in slab order."""
        return _combine(self.e[0], [e.diag_partials(r_bar_max) for e in self.e])[1]

    def close(self):
        for e in self.e:
            e.close()


class SlabRank:
    """This process's slab of a grid split over the ranks of a process group,
    rank r owning phi slab r.  Ghost planes travel by send/recv (tagged by
    direction and posted in the same order on every rank, so that two ranks
    that are each other's left and right neighbours still match them); the
    CFL minima are combined by a MIN all-reduce."""

    TAG_RIGHTWARD, TAG_LEFTWARD = 1, 2

    def __init__(self, engine, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.e = engine
        self.rank = dist.get_rank(group)
        self.R = dist.get_world_size(group)
        self.left, self.right = (self.rank - 1) % self.R, (self.rank + 1) % self.R
        if group is not None:
            self.left = dist.get_global_rank(group, self.left)
            self.right = dist.get_global_rank(group, self.right)
        mk = lambda: torch.empty(engine.plane_numel, dtype=engine.dtype, device=engine.device)
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()
        self.dtd_buf = torch.empty(3, dtype=torch.float64, device=engine.device)

    def set_state(self, P, U, t, dt):
        """P, U: the whole grid's state (every rank holds the same); this
        rank keeps its slab."""
        with _stream_of(self.e):
            self.e.set_state(split_phi(P, self.R, self.rank), split_phi(U, self.R, self.rank), t, dt)
        self.exchange(0)

    def exchange(self, which):
        e, dist = self.e, self.dist
        e.pack(which, 0, self.send_lo)
        e.pack(which, 1, self.send_hi)
        if self.R == 1:
            e.unpack(which, 0, self.send_hi)
            e.unpack(which, 1, self.send_lo)
            return
        with _stream_of(e):
            ops = [dist.P2POp(dist.isend, self.send_hi, self.right, self.group, self.TAG_RIGHTWARD),
                   dist.P2POp(dist.isend, self.send_lo, self.left, self.group, self.TAG_LEFTWARD),
                   dist.P2POp(dist.irecv, self.recv_lo, self.left, self.group, self.TAG_RIGHTWARD),
                   dist.P2POp(dist.irecv, self.recv_hi, self.right, self.group, self.TAG_LEFTWARD)]
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        e.unpack(which, 0, self.recv_lo)
        e.unpack(which, 1, self.recv_hi)

    def step(self, nsteps=1):
        e = self.e
        for _ in range(nsteps):
            e.stage(0)
            e.dtd(self.dtd_buf)
            self.exchange(1)
            e.stage(1)
            self.exchange(0)
            if self.R > 1:
                with _stream_of(e):
                    self.dist.all_reduce(self.dtd_buf, op=self.dist.ReduceOp.MIN, group=self.group)
            e.finish(self.dtd_buf)

    def _gathered(self, r_bar_max):
        """Every rank's partial vector, gathered on the device in rank order
        and combined by the library (the same bits on every rank)."""
        buf = self.e.diag_partials(r_bar_max)
        with _stream_of(self.e):
            parts = [torch.empty_like(buf) for _ in range(self.R)]
            self.dist.all_gather(parts, buf, group=self.group)
        return _combine(self.e, parts)

    def diagnostics(self, r_bar_max=80.0):
        """The whole grid's diagnostics on every rank."""
        return self._gathered(r_bar_max)[0]

    def barycentric_radius(self, r_bar_max=80.0):
        return self._gathered(r_bar_max)[1]


# ------------------------------------------------------------ theta slabs
#
# The split of the paper's multi-GPU runs (Section 3) in theta, for
# axisymmetric grids (n3 = 1), which cannot be split in phi.  Slab r of R owns
# the active rows [r n2/R, (r+1) n2/R) of the whole grid (grid parameters j0,
# n2_total) and builds the metric of its own rows from their global X2
# positions, so its tables are bit for bit the whole grid's.  One step:
#   for each stage st (Eq. 25, then Eq. 26):
#     1. every slab runs the fluxes, flux-CT, update and inversion;
#     2. fixups (Eq. 33): while some slab has a failed zone and fewer than
#        fix_maxsweep sweeps ran, exchange the edge rows that a sweep reads
#        across a slab face (five primitives and the failure flags), then
#        run one sweep on every slab;
#     3. every slab fills its own boundaries (poles, radial), then the NG = 3
#        ghost rows of its inner sides are exchanged;
#   the CFL minima of the predictor are reduced as for phi slabs.
# Every value a slab reads across its faces is the one the whole grid reads
# there, so the decomposed step is the undecomposed one bit for bit.


def theta_grid(base: G.GridParams, R: int, r: int) -> G.GridParams:
    """Grid parameters of theta slab r of R (n2 / R rows starting at row
    r n2 / R of the whole grid; at least 4 rows)."""
    if R < 1 or base.n2 % R:
        raise ValueError(f"n2 = {base.n2} does not split into {R} slabs")
    n2 = base.n2 // R
    if n2 < 4:
        raise ValueError(f"theta slabs of {n2} < 4 rows")
    g = G.GridParams.from_buffer_copy(base)
    g.n2, g.j0, g.n2_total = n2, r * n2, base.n2
    return g


def split_theta(x, R: int, r: int):
    """Slab r's part of a (fields, n1, n2, n3) array (numpy or torch), contiguous."""
    n2 = x.shape[2] // R
    part = x[:, :, r * n2:(r + 1) * n2]
    return part.contiguous() if isinstance(x, torch.Tensor) else part.copy(order="C")


class CtxTheta:
    """ThetaEngine over one grmhd context that is a theta slab.  Every call
    is asynchronous on the context's stream (`stream`)."""

    def __init__(self, ctx: G.Context, stream: torch.cuda.Stream):
        if not (ctx.grid.n2_total > ctx.grid.n2):
            raise ValueError("a theta slab context needs n2_total > n2")
        self.ctx = ctx
        self.stream = stream
        self.device = torch.device("cuda", ctx.grid.device)
        self.dtype = torch.float64 if ctx.grid.precision == G.FP64 else torch.float32
        esz = 8 if self.dtype == torch.float64 else 4
        self.row_numel = G.x2_row_bytes(ctx, 0) // esz
        self.fix_numel = G.x2_row_bytes(ctx, 1) // esz
        self.fix_maxsweep = ctx.phys.fix_maxsweep

    @classmethod
    def create(cls, grid: G.GridParams, phys: G.PhysParams, a: float, stream: torch.cuda.Stream):
        g = G.GridParams.from_buffer_copy(grid)
        g.stream = stream.cuda_stream
        ctx = G.init_grid(g, phys)
        G.set_metric(ctx, a, g.metric)
        return cls(ctx, stream)

    def set_state(self, P, U, t, dt):
        G.set_state(self.ctx, P, U, t, dt)

    def get_state(self):
        return G.get_state(self.ctx)

    def diagnostics(self):
        return G.diagnostics(self.ctx)

    def diag_partials(self, r_bar_max):
        out = torch.empty(G.DIAG_NPART, dtype=torch.float64, device=self.device)
        G.diag_partials(self.ctx, r_bar_max, out)  # on the context stream
        return out

    def diag_combine(self, parts):
        return G.diag_combine(self.ctx, parts)

    def stage_update(self, st):
        G.stage_update(self.ctx, st)

    def dtd(self, out, accumulate=False):
        G.step_dtd(self.ctx, out, accumulate)

    def fail_count(self, acc):
        G.fail_count(self.ctx, acc)

    def fix_sweep(self, st, acc):
        G.fix_sweep(self.ctx, st, acc)

    def fix_end(self, st, nsweeps):
        G.fix_end(self.ctx, st, nsweeps)

    def stage_bc(self, st):
        G.stage_bc(self.ctx, st)

    def finish(self, dtd):
        G.finish_step(self.ctx, dtd)

    def pack(self, kind, which, side, buf):
        G.x2_pack(self.ctx, kind, which, side, buf)

    def unpack(self, kind, which, side, buf):
        G.x2_unpack(self.ctx, kind, which, side, buf)

    def close(self):
        self.ctx.close()


def _theta_sides(R: int, r: int, periodic: bool):
    """(low, high) neighbour slab of slab r, None at a pole or closed side."""
    lo = (r - 1) % R if (r > 0 or periodic) else None
    hi = (r + 1) % R if (r < R - 1 or periodic) else None
    return lo, hi


class ThetaRing:
    """All theta slabs of one grid on one device, in theta order, sharing one
    stream.  `periodic`: the whole grid is periodic in X2 (a flat box), so
    the first and last slabs are neighbours.

    Library slabs (CtxTheta) run each stage's fixup loop on the device
    (grmhd_theta_ring_fix: nothing read on the host), so a step is a fixed
    sequence of device work, captured once in a CUDA graph and replayed (as
    SlabRing's, drop_graph() after a change of a context's grid record).
    device_fix=False, or other engines, run the loop from the host over the
    per-slab calls (fail counts read on the host, kind-1 row exchanges)."""

    ROWS, FIX = 0, 1  # the two exchanges: NG ghost rows, a fixup sweep's edge row

    def __init__(self, engines, periodic: bool = False, device_fix: bool = True):
        self.e = list(engines)
        self.periodic = periodic
        e0 = self.e[0]
        R = len(self.e)
        self.nb = [_theta_sides(R, r, periodic) for r in range(R)]
        mk = lambda n: [torch.empty(n, dtype=e.dtype, device=e.device) for e in self.e]
        self.buf = {self.ROWS: (mk(e0.row_numel), mk(e0.row_numel)),
                    self.FIX: (mk(e0.fix_numel), mk(e0.fix_numel))}
        self.dtd_buf = torch.empty(3, dtype=torch.float64, device=e0.device)
        self.count = torch.zeros(1, dtype=torch.int64, device=e0.device)
        self.fix_maxsweep = e0.fix_maxsweep
        streams = {id(getattr(e, "stream", None)) for e in self.e}
        self.device_fix = device_fix and all(isinstance(e, CtxTheta) for e in self.e) and len(streams) == 1
        self._nsw = torch.zeros(2, dtype=torch.int32, device=e0.device) if self.device_fix else None
        self._sweeps = []  # host loop: fixup sweeps of each stage of the last step
        self._graph = None

    @classmethod
    def create(cls, grid: G.GridParams, phys: G.PhysParams, R: int, a: float, stream=None, periodic=False,
               device_fix=True):
        stream = stream or torch.cuda.Stream(device=grid.device)
        return cls([CtxTheta.create(theta_grid(grid, R, r), phys, a, stream) for r in range(R)], periodic,
                   device_fix)

    @property
    def sweeps(self):
        """Fixup sweeps of each stage of the last step."""
        if self.device_fix:
            with _stream_of(self.e[0]):
                return [int(v) for v in self._nsw.cpu()]
        return list(self._sweeps)

    def set_state(self, P, U, t, dt):
        R = len(self.e)
        for r, e in enumerate(self.e):
            with _stream_of(e):
                e.set_state(split_theta(P, R, r), split_theta(U, R, r), t, dt)
        self.exchange(self.ROWS, 0)

    def exchange(self, kind, which):
        """Pack every slab's edge rows, then unpack each into its
        neighbours' ghost rows (one stream, so ordered)."""
        lo, hi = self.buf[kind]
        for r, e in enumerate(self.e):
            e.pack(kind, which, 0, lo[r])
            e.pack(kind, which, 1, hi[r])
        for r, e in enumerate(self.e):
            left, right = self.nb[r]
            if left is not None:
                e.unpack(kind, which, 0, hi[left])
            if right is not None:
                e.unpack(kind, which, 1, lo[right])

    def _count(self, fn):
        self.count.zero_()
        for e in self.e:
            fn(e)
        return int(self.count.item())

    def _fixups(self, st, out):
        if self.device_fix:
            G.theta_ring_fix([e.ctx for e in self.e], st, self._nsw[st:st + 1])
            for e in self.e:
                e.stage_bc(st)
            return
        left = self._count(lambda e: e.fail_count(self.count))
        n = 0
        while left > 0 and n < self.fix_maxsweep:
            self.exchange(self.FIX, out)
            left = self._count(lambda e: e.fix_sweep(st, self.count))
            n += 1
        self._sweeps.append(n)
        for e in self.e:
            e.fix_end(st, n)
            e.stage_bc(st)

    def _step_once(self):
        self._sweeps = []
        for st in (0, 1):
            out = 1 if st == 0 else 0  # the stage's output buffer
            for r, e in enumerate(self.e):
                e.stage_update(st)
                if st == 0:
                    e.dtd(self.dtd_buf, accumulate=r > 0)
            self._fixups(st, out)
            self.exchange(self.ROWS, out)
        for e in self.e:
            e.finish(self.dtd_buf)

    def step(self, nsteps=1, graph=True):
        """nsteps RK2 steps of the whole grid; graph=False launches every
        kernel from the host."""
        s = self.e[0].stream if hasattr(self.e[0], "stream") else None
        if not (graph and self.device_fix):
            with _stream_of(self.e[0]):
                for _ in range(nsteps):
                    self._step_once()
            return
        if self._graph is None:
            self._graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self._graph, stream=s):
                self._step_once()
        with torch.cuda.stream(s):
            for _ in range(nsteps):
                self._graph.replay()

    def drop_graph(self):
        self._graph = None

    def diagnostics(self, r_bar_max=80.0):
        return _combine(self.e[0], [e.diag_partials(r_bar_max) for e in self.e])[0]

    def barycentric_radius(self, r_bar_max=80.0):
        return _combine(self.e[0], [e.diag_partials(r_bar_max) for e in self.e])[1]

    def close(self):
        for e in self.e:
            e.close()


class ThetaRank:
    """This process's theta slab of a grid split over the ranks of a
    process group, rank r owning slab r.  Edge rows travel by send/recv
    (tags by direction, as for phi slabs); the failure counts that decide
    the fixup sweeps and the CFL minima are all-reduced (SUM, MIN)."""

    TAG_UP, TAG_DOWN = 3, 4

    def __init__(self, engine, group=None, periodic: bool = False):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.e = engine
        self.rank = dist.get_rank(group)
        self.R = dist.get_world_size(group)
        lo, hi = _theta_sides(self.R, self.rank, periodic)
        if group is not None:
            lo = dist.get_global_rank(group, lo) if lo is not None else None
            hi = dist.get_global_rank(group, hi) if hi is not None else None
        self.left, self.right = lo, hi
        mk = lambda n: torch.empty(n, dtype=engine.dtype, device=engine.device)
        self.buf = {k: (mk(n), mk(n), mk(n), mk(n))
                    for k, n in ((ThetaRing.ROWS, engine.row_numel), (ThetaRing.FIX, engine.fix_numel))}
        self.dtd_buf = torch.empty(3, dtype=torch.float64, device=engine.device)
        self.count = torch.zeros(1, dtype=torch.int64, device=engine.device)
        self.fix_maxsweep = engine.fix_maxsweep
        self.sweeps = []

    def set_state(self, P, U, t, dt):
        with _stream_of(self.e):
            self.e.set_state(split_theta(P, self.R, self.rank), split_theta(U, self.R, self.rank), t, dt)
        self.exchange(ThetaRing.ROWS, 0)

    def exchange(self, kind, which):
        e, dist = self.e, self.dist
        send_lo, send_hi, recv_lo, recv_hi = self.buf[kind]
        e.pack(kind, which, 0, send_lo)
        e.pack(kind, which, 1, send_hi)
        if self.R == 1:  # periodic single slab: its own far rows
            if self.left is not None:
                e.unpack(kind, which, 0, send_hi)
                e.unpack(kind, which, 1, send_lo)
            return
        ops = []
        if self.right is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, self.right, self.group, self.TAG_UP))
        if self.left is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, self.left, self.group, self.TAG_DOWN))
        if self.left is not None:
            ops.append(dist.P2POp(dist.irecv, recv_lo, self.left, self.group, self.TAG_UP))
        if self.right is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, self.right, self.group, self.TAG_DOWN))
        with _stream_of(e):
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if self.left is not None:
            e.unpack(kind, which, 0, recv_lo)
        if self.right is not None:
            e.unpack(kind, which, 1, recv_hi)

    def _count(self, fn):
        with _stream_of(self.e):
            self.count.zero_()
            fn()
            if self.R > 1:
                self.dist.all_reduce(self.count, op=self.dist.ReduceOp.SUM, group=self.group)
            return int(self.count.item())

    def step(self, nsteps=1):
        e = self.e
        for _ in range(nsteps):
            self.sweeps = []
            for st in (0, 1):
                out = 1 if st == 0 else 0
                e.stage_update(st)
                if st == 0:
                    e.dtd(self.dtd_buf)
                left = self._count(lambda: e.fail_count(self.count))
                n = 0
                while left > 0 and n < self.fix_maxsweep:
                    self.exchange(ThetaRing.FIX, out)
                    left = self._count(lambda: e.fix_sweep(st, self.count))
                    n += 1
                self.sweeps.append(n)
                e.fix_end(st, n)
                e.stage_bc(st)
                self.exchange(ThetaRing.ROWS, out)
            if self.R > 1:
                with _stream_of(e):
                    self.dist.all_reduce(self.dtd_buf, op=self.dist.ReduceOp.MIN, group=self.group)
            e.finish(self.dtd_buf)

    _gathered = SlabRank._gathered

    def diagnostics(self, r_bar_max=80.0):
        return self._gathered(r_bar_max)[0]

    def barycentric_radius(self, r_bar_max=80.0):
        return self._gathered(r_bar_max)[1]


__all__ = ["NG", "slab_grid", "split_phi", "CtxSlab", "SlabRing", "SlabRank",
           "theta_grid", "split_theta", "CtxTheta", "ThetaRing", "ThetaRank"]
