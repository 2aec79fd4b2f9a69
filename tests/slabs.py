"""A phi-slab decomposition of the step (one ghost exchange per stage, a
global minimum for dt), run on the oracle: the host logic a multi-GPU run
follows, checked against the undecomposed grid.

Each slab r of R owns the active phi zones [r n3/R, (r+1) n3/R) and a copy of
the (r, theta) metric; after every stage its NG = 3 X3 ghost planes on each
side are the neighbours' outermost active planes (periodic in phi), taken
after the neighbours' own X1/X2 boundary fill.  The predictor's per-direction
CFL minima are reduced over slabs and then combined by Eq. 27.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O

NG = O.NG


def slab_params(base: O.Params, r: int, R: int) -> O.Params:
    """Parameters of slab r: n3 / R phi zones, X3 ghosts external.  The
    step never uses a slab's phi position (the metric does not depend on
    phi), only dX3, so the slab's X3 range starts at 0 and spans
    (n3 / R) 2 pi / n3: for power-of-two slab widths dX3 = 2 pi / n3 exactly,
    as in the undecomposed grid."""
    d = {name: getattr(base, name) for name, _ in O.Params._fields_}
    n3 = base.n3 // R
    d.update(n3=n3, bc3=O.BC_EXTERNAL, x3min=0.0, x3max=n3 * (2.0 * math.pi / base.n3))
    return O.Params(**d)


def split_state(P, U, R):
    n3 = P.shape[3] // R
    return [(np.ascontiguousarray(P[..., r * n3:(r + 1) * n3]), np.ascontiguousarray(U[..., r * n3:(r + 1) * n3]))
            for r in range(R)]


def ghost_planes_from(left, right, n3, which):
    """The ghost planes of a slab: k = -2, -1 from its left neighbour's
    k = n3-2, n3-1 and k = n3, n3+1 from its right neighbour's k = 0, 1."""
    lo = [left.xplane(which, n3 - NG + g) for g in range(NG)]
    hi = [right.xplane(which, g) for g in range(NG)]
    return lo, hi


def exchange(slabs, which):
    n3 = slabs[0].shape[2]
    R = len(slabs)
    planes = [ghost_planes_from(slabs[(r - 1) % R], slabs[(r + 1) % R], n3, which) for r in range(R)]
    for r, (lo, hi) in enumerate(planes):
        for g in range(NG):
            slabs[r].set_xplane(which, -NG + g, lo[g])
            slabs[r].set_xplane(which, n3 + g, hi[g])


def make_slabs(base: O.Params, P, U, t, dt, R):
    slabs = [O.Grid(slab_params(base, r, R)) for r in range(R)]
    for g, (Ps, Us) in zip(slabs, split_state(P, U, R)):
        g.set_state(Ps, Us, t, dt)
    exchange(slabs, 0)
    return slabs


def step_slabs(slabs):
    cand, status = [], 0
    for g in slabs:
        _, st = g.stage0()
        cand.append(g.last_dtd())
        status = status or st
    exchange(slabs, 1)
    for g in slabs:
        status = g.stage1() or status
    exchange(slabs, 0)
    # Eq. 27 over the whole grid: per-direction minima first, then combined
    dt = O.combine_dt(np.min(np.array(cand), axis=0))
    for g in slabs:
        g.set_dt(dt)
    return status


def gather(slabs):
    parts = [g.get_state() for g in slabs]
    P = np.concatenate([p[0] for p in parts], axis=3)
    U = np.concatenate([p[1] for p in parts], axis=3)
    return P, U, parts[0][2], parts[0][3]


# ---------------------------------------------------- combined diagnostics
# The layout of the library's partial vector (grmhd_diag_partials) filled from
# an oracle slab, and its combination written out on the oracle side, so that
# the product's slab drivers run over oracle slabs on the CPU.
DIAG_NPART = 26
_COUNTERS = ("nr_iters", "n_nr", "n_brent", "n_entropy", "n_entropy_beta", "n_fail", "n_floor", "n_ceil",
             "n_gcap", "n_fixed", "fix_sweeps", "n_steps", "n_learned")


def oracle_partials(g, r_bar_max):
    import torch
    d = g.diagnostics()
    v = np.zeros(DIAG_NPART)
    v[0:5] = [d["mdot"], d["phib"], d["edot"], d["ldot"], d["divb_max"]]
    if r_bar_max > 0.0 and g.p.metric == O.KERR_MKS:
        _, den, num = g.barycentric(r_bar_max)
        v[5:7] = [num, den]
    v[7:9] = [d["t"], d["dt"]]
    for c, k in enumerate(_COUNTERS):
        v[9 + c] = d.get(k, 0)
    return torch.tensor(v, dtype=torch.float64)


def oracle_combine(parts):
    """Sum in row order, div B and sweeps by the largest, steps/t/dt of the
    first row; Eq. 42, the efficiency and the Eq. 43 quotient of the sums."""
    P = np.asarray(parts.cpu().numpy(), dtype=np.float64)
    v = P[0].copy()
    for p in P[1:]:
        v[0:4] += p[0:4]
        v[4] = max(v[4], p[4])
        v[5:7] += p[5:7]
        for c, k in enumerate(_COUNTERS):
            if k == "fix_sweeps":
                v[9 + c] = max(v[9 + c], p[9 + c])
            elif k != "n_steps":
                v[9 + c] += p[9 + c]
    mdot = v[0]
    d = {"t": v[7], "dt": v[8], "mdot": mdot, "phib": v[1], "edot": v[2], "ldot": v[3], "divb_max": v[4],
         "PhiB": v[1] / np.sqrt(abs(mdot)) if mdot != 0.0 else 0.0,
         "eta": (v[2] - mdot) / abs(mdot) if mdot != 0.0 else 0.0, "disk_mass": 0.0, "disk_eb": 0.0}
    for c, k in enumerate(_COUNTERS):
        d[k] = int(v[9 + c])
    bary = (v[5] / v[6] if v[6] > 0.0 else 0.0, v[6], v[5])
    return d, bary


class OracleSlab:
    """The SlabEngine interface of paper_2205_02484_gb300.decomp over one
    oracle slab, so that the product's slab drivers (their exchange order,
    tags and dt reduction) can run on the CPU with the oracle doing the
    stages.  Buffers are CPU float64 tensors in the [NG][8][N1][N2] layout."""

    def __init__(self, params: O.Params):
        import torch
        self.g = O.Grid(params)
        self.n3 = params.n3
        self.device = torch.device("cpu")
        self.dtype = torch.float64
        self.plane_numel = NG * O.NP * self.g.N[0] * self.g.N[1]

    def set_state(self, P, U, t, dt):
        self.g.set_state(np.asarray(P), np.asarray(U), t, dt)

    def get_state(self):
        return self.g.get_state()

    def diagnostics(self):
        return self.g.diagnostics()

    def barycentric_sums(self, r_bar_max):
        _, den, num = self.g.barycentric(r_bar_max)
        return num, den

    def diag_partials(self, r_bar_max):
        return oracle_partials(self.g, r_bar_max)

    def diag_combine(self, parts):
        return oracle_combine(parts)

    def stage(self, st):
        if st == 0:
            assert self.g.stage0()[1] == 0
        else:
            assert self.g.stage1() == 0

    def dtd(self, out, accumulate=False):
        import torch
        v = torch.from_numpy(self.g.last_dtd())
        out.copy_(torch.minimum(out, v) if accumulate else v)

    def finish(self, dtd):
        # the oracle's corrector has already advanced t by the old dt
        self.g.set_dt(O.combine_dt(dtd.numpy()))

    def _ks(self, side, ghost):
        if ghost:
            return range(-NG, 0) if side == 0 else range(self.n3, self.n3 + NG)
        return range(0, NG) if side == 0 else range(self.n3 - NG, self.n3)

    def pack(self, which, side, buf):
        import torch
        planes = np.stack([self.g.xplane(which, k) for k in self._ks(side, False)])
        buf.copy_(torch.from_numpy(planes.reshape(-1)))

    def unpack(self, which, side, buf):
        planes = buf.numpy().reshape(NG, O.NP, self.g.N[0], self.g.N[1])
        for g_, k in enumerate(self._ks(side, True)):
            self.g.set_xplane(which, k, planes[g_])


# ------------------------------------------------------------ theta slabs
# A theta-slab decomposition (the split of the paper's multi-GPU runs,
# Section 3; here for axisymmetric grids): slab r owns the active rows
# [r n2/R, (r+1) n2/R) and builds its own rows of the metric; after every
# stage its NG = 3 X2 ghost rows on an inner side are the neighbour's edge
# rows.  The fixups of Eq. 33 average across a slab face, so before every
# sweep each slab receives the neighbour's current edge row (five
# primitives and the failure flags), and the sweeps run while any slab has a
# failed zone.


def theta_params(base: O.Params, r: int, R: int) -> O.Params:
    d = {name: getattr(base, name) for name, _ in O.Params._fields_}
    n2 = base.n2 // R
    d.update(n2=n2, j0=r * n2, n2_total=base.n2)
    return O.Params(**d)


def split_theta(P, U, R):
    n2 = P.shape[2] // R
    return [(np.ascontiguousarray(P[:, :, r * n2:(r + 1) * n2]), np.ascontiguousarray(U[:, :, r * n2:(r + 1) * n2]))
            for r in range(R)]


def _theta_neighbours(R, periodic):
    """(left, right) slab of each slab, None at a pole / closed side."""
    out = []
    for r in range(R):
        lo = (r - 1) % R if (r > 0 or periodic) else None
        hi = (r + 1) % R if (r < R - 1 or periodic) else None
        out.append((lo, hi))
    return out


def exchange_rows(slabs, which, periodic=False):
    n2 = slabs[0].shape[1]
    nb = _theta_neighbours(len(slabs), periodic)
    rows = []
    for r, (lo, hi) in enumerate(nb):
        rows.append(([slabs[lo].yrow(which, n2 - NG + g) for g in range(NG)] if lo is not None else None,
                     [slabs[hi].yrow(which, g) for g in range(NG)] if hi is not None else None))
    for r, (lo, hi) in enumerate(rows):
        if lo is not None:
            for g in range(NG):
                slabs[r].set_yrow(which, -NG + g, lo[g])
        if hi is not None:
            for g in range(NG):
                slabs[r].set_yrow(which, n2 + g, hi[g])


def exchange_fixrows(slabs, which, periodic=False):
    n2 = slabs[0].shape[1]
    nb = _theta_neighbours(len(slabs), periodic)
    rows = [(slabs[lo].fixrow(which, n2 - 1) if lo is not None else None,
             slabs[hi].fixrow(which, 0) if hi is not None else None) for lo, hi in nb]
    for r, (lo, hi) in enumerate(rows):
        if lo is not None:
            slabs[r].set_fixrow(which, -1, lo)
        if hi is not None:
            slabs[r].set_fixrow(which, n2, hi)


def make_theta_slabs(base: O.Params, P, U, t, dt, R, periodic=False):
    slabs = [O.Grid(theta_params(base, r, R)) for r in range(R)]
    for g, (Ps, Us) in zip(slabs, split_theta(P, U, R)):
        g.set_state(Ps, Us, t, dt)
    exchange_rows(slabs, 0, periodic)
    return slabs


def step_theta_slabs(slabs, periodic=False):
    """One RK2 step of the decomposed grid; returns the fixup status (0, or
    -1 if some zone stayed failed) and the number of sweeps of each stage."""
    maxsweep = slabs[0].p.fix_maxsweep
    cand, status, sweeps = [], 0, []
    for st in (0, 1):
        which = 1 if st == 0 else 0  # the stage's output buffer
        for g in slabs:
            g.stage_update(st)
            if st == 0:
                cand.append(g.last_dtd())
        left, n = sum(g.fail_count() for g in slabs), 0
        while left > 0 and n < maxsweep:
            exchange_fixrows(slabs, which, periodic)
            left = sum(g.fix_sweep(st) for g in slabs)
            n += 1
        status = status or (-1 if left > 0 else 0)
        sweeps.append(n)
        for g in slabs:
            g.fix_end(n)
            g.stage_bc(st)
        exchange_rows(slabs, which, periodic)
    dt = O.combine_dt(np.min(np.array(cand), axis=0))
    for g in slabs:
        g.set_dt(dt)
    return status, sweeps


def gather_theta(slabs):
    parts = [g.get_state() for g in slabs]
    P = np.concatenate([p[0] for p in parts], axis=2)
    U = np.concatenate([p[1] for p in parts], axis=2)
    return P, U, parts[0][2], parts[0][3]


class OracleThetaSlab:
    """The ThetaEngine interface of paper_2205_02484_gb300.decomp over one
    oracle theta slab (CPU float64 tensors; ghost rows [NG][8][N1][N3],
    fixup rows [6][n1][n3])."""

    def __init__(self, params: O.Params):
        import torch
        self.g = O.Grid(params)
        self.n2 = params.n2
        self.device = torch.device("cpu")
        self.dtype = torch.float64
        self.row_numel = NG * O.NP * self.g.N[0] * self.g.N[2]
        self.fix_numel = 6 * params.n1 * params.n3
        self.fix_maxsweep = params.fix_maxsweep

    def set_state(self, P, U, t, dt):
        self.g.set_state(np.asarray(P), np.asarray(U), t, dt)

    def get_state(self):
        return self.g.get_state()

    def diagnostics(self):
        return self.g.diagnostics()

    def barycentric_sums(self, r_bar_max):
        _, den, num = self.g.barycentric(r_bar_max)
        return num, den

    def diag_partials(self, r_bar_max):
        return oracle_partials(self.g, r_bar_max)

    def diag_combine(self, parts):
        return oracle_combine(parts)

    def stage_update(self, st):
        self.g.stage_update(st)

    def dtd(self, out, accumulate=False):
        import torch
        v = torch.from_numpy(self.g.last_dtd())
        out.copy_(torch.minimum(out, v) if accumulate else v)

    def fail_count(self, acc):
        acc += self.g.fail_count()

    def fix_sweep(self, st, acc):
        acc += self.g.fix_sweep(st)

    def fix_end(self, st, nsweeps):
        self.g.fix_end(nsweeps)

    def stage_bc(self, st):
        self.g.stage_bc(st)

    def finish(self, dtd):
        self.g.set_dt(O.combine_dt(dtd.numpy()))

    def _rows(self, kind, side, ghost):
        n = NG if kind == 0 else 1
        if ghost:
            return range(-n, 0) if side == 0 else range(self.n2, self.n2 + n)
        return range(0, n) if side == 0 else range(self.n2 - n, self.n2)

    def pack(self, kind, which, side, buf):
        import torch
        get = self.g.yrow if kind == 0 else self.g.fixrow
        rows = np.stack([get(which, j) for j in self._rows(kind, side, False)])
        buf.copy_(torch.from_numpy(rows.reshape(-1)))

    def unpack(self, kind, which, side, buf):
        put = self.g.set_yrow if kind == 0 else self.g.set_fixrow
        shape = (NG, O.NP, self.g.N[0], self.g.N[2]) if kind == 0 else (1, 6, self.g.p.n1, self.g.p.n3)
        rows = buf.numpy().reshape(shape)
        for g_, j in enumerate(self._rows(kind, side, True)):
            put(which, j, rows[g_])
