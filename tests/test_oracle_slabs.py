"""The phi-slab decomposition of the step (tests/slabs.py) reproduces the
undecomposed oracle bit for bit: in-process with 2 and 4 slabs, and as 2 and
4 gloo ranks driven by the library's rank driver (SlabRank), which exchanges
ghost planes with send/recv and reduces the per-direction CFL minima with an
all-reduce, the oracle doing each slab's stages."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from tests import slabs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _base(**kw):
    return O.default_params(n1=20, n2=16, n3=8, gam=13.0 / 9.0, r_out=40.0, **kw)


def _reference_grid(steps):
    g = O.Grid(_base())
    g.init_torus(pert_amp=0.04, seed=5)
    for _ in range(steps):
        assert g.step() == 0
    return g


def _check_combined(dr, df):
    """Slab diagnostics combined vs the undecomposed grid's: the horizon
    integrals (Eqs. 38-41) to rounding, the counters exactly, div B (Eq. 24)
    over the corners inside the slabs, a subset of the grid's corners."""
    for k in ("mdot", "phib", "PhiB", "edot", "ldot", "eta"):
        assert dr[k] == pytest.approx(df[k], rel=1e-12), k
    for k in ("n_nr", "n_brent", "n_fail", "n_floor", "n_ceil", "n_fixed"):
        assert dr[k] == df[k], k
    assert 0.0 < dr["divb_max"] <= df["divb_max"]


def _reference(steps):
    g = O.Grid(_base())
    g.init_torus(pert_amp=0.04, seed=5)
    P0, U0, t0, dt0 = g.get_state()
    for _ in range(steps):
        assert g.step() == 0
    return (P0, U0, t0, dt0), g.get_state()


@pytest.mark.parametrize("R", [2, 4])
def test_slabs_reproduce_the_undecomposed_step(R):
    (P0, U0, t0, dt0), (Pr, Ur, tr, dtr) = _reference(4)
    slabs = S.make_slabs(_base(), P0, U0, t0, dt0, R)
    for _ in range(4):
        assert S.step_slabs(slabs) == 0
    P, U, t, dt = S.gather(slabs)
    assert t == tr and dt == dtr
    assert np.array_equal(P, Pr)
    assert np.array_equal(U, Ur)
    import torch
    parts = torch.stack([S.oracle_partials(g, 0.0) for g in slabs])
    _check_combined(S.oracle_combine(parts)[0], _reference_grid(4).diagnostics())


def test_slabs_with_ppm_and_cylindrification():
    """PPM faces (all NG = 3 exchanged planes read) on a cylindrified grid:
    2 phi slabs reproduce the undecomposed oracle bit for bit."""
    kw = dict(recon=O.PPM, cyl_r=1.8, cyl_dx2=0.3)
    g = O.Grid(_base(**kw))
    g.init_torus(pert_amp=0.04, seed=5)
    P0, U0, t0, dt0 = g.get_state()
    for _ in range(3):
        assert g.step() == 0
    slabs = S.make_slabs(_base(**kw), P0, U0, t0, dt0, 2)
    for _ in range(3):
        assert S.step_slabs(slabs) == 0
    P, U, t, dt = S.gather(slabs)
    Pr, Ur, tr, dtr = g.get_state()
    assert (t, dt) == (tr, dtr)
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)


@pytest.mark.parametrize("R", [2, 4])
def test_slab_ring_over_oracle_slabs(R):
    """SlabRing (the single-device driver) with the oracle as its engines:
    they have no CUDA stream, so the ring steps them by host calls (the graph
    form is for library slabs) and reproduces the undecomposed oracle."""
    pytest.importorskip("torch")
    from paper_2205_02484_gb300.decomp import SlabRing
    (P0, U0, t0, dt0), (Pr, Ur, tr, dtr) = _reference(3)
    ring = SlabRing([S.OracleSlab(S.slab_params(_base(), r, R)) for r in range(R)])
    assert not ring._capturable
    ring.set_state(P0, U0, t0, dt0)
    ring.step(3)
    P = np.concatenate([e.get_state()[0] for e in ring.e], axis=3)
    U = np.concatenate([e.get_state()[1] for e in ring.e], axis=3)
    assert ring.e[0].get_state()[2:] == (tr, dtr)
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)
    _check_combined(ring.diagnostics(), _reference_grid(3).diagnostics())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, steps, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2205_02484_gb300.decomp import SlabRank
    from tests import slabs as S2
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = _base()
    g = O.Grid(base)
    g.init_torus(pert_amp=0.04, seed=5)
    P0, U0, t0, dt0 = g.get_state()
    # the product's rank driver, with the oracle doing the stages
    slab = SlabRank(S2.OracleSlab(S2.slab_params(base, rank, world)))
    slab.set_state(P0, U0, t0, dt0)
    slab.step(steps)
    P, U, t, dt = slab.e.get_state()
    diag = slab.diagnostics()
    diag["bary"] = slab.barycentric_radius(30.0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (P, U, t, dt, diag))
    dist.destroy_process_group()
    if rank == 0:
        out.put(gathered)


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_reproduce_the_undecomposed_step(world):
    """world 2: each rank is both neighbours of the other (the send/recv
    matching case); world 4: distinct neighbours."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, 3, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, (Pr, Ur, tr, dtr) = _reference(3)
    P = np.concatenate([g[0] for g in gathered], axis=3)
    U = np.concatenate([g[1] for g in gathered], axis=3)
    assert gathered[0][2] == tr and gathered[0][3] == dtr
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)
    # every rank holds the whole grid's diagnostics
    assert all(g[4] == gathered[0][4] for g in gathered)
    ref = _reference_grid(3)
    _check_combined(gathered[0][4], ref.diagnostics())
    for x, y in zip(gathered[0][4]["bary"], ref.barycentric(30.0)):
        assert x == pytest.approx(y, rel=1e-13)
