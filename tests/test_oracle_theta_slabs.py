"""The theta-slab decomposition of the step reproduces the undecomposed
oracle bit for bit: the in-process ring of tests/slabs.py and the library's
drivers (ThetaRing in one process, ThetaRank as gloo ranks), the oracle doing
each slab's stage parts.  A block of zones made to fail straddles a slab face
in both stages, so the fixup sweeps of Eq. 33 read across the face and need
several rounds."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from tests import slabs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _base(n3=1, **kw):
    return O.default_params(n1=24, n2=24, n3=n3, gam=13.0 / 9.0, r_out=40.0, **kw)


def _spoil(U, rows, cols):
    """Make the inversion of a block of zones fail in both stages (negative
    conserved density, C2P_FAIL_D): the predictor's fixups repair P-hat, the
    corrector's repair P and rebuild U from it."""
    U = U.copy()
    for j in rows:
        for i in cols:
            U[0, i, j, :] = -1.0
    return U


def _torus_start(n3=1, R=2, **kw):
    g = O.Grid(_base(n3, **kw))
    g.init_torus(pert_amp=0.04, seed=5)
    P0, U0, t0, dt0 = g.get_state()
    b = 24 // R  # the first inner slab face
    return P0, _spoil(U0, range(b - 3, b + 3), range(8, 15)), t0, dt0


def _undecomposed(base, state, steps):
    g = O.Grid(base)
    g.set_state(*state)
    for _ in range(steps):
        assert g.step() == 0
    return g


def _check_combined(dr, df, exact_sweeps=True):
    for k in ("mdot", "phib", "PhiB", "edot", "ldot", "eta"):
        assert dr[k] == pytest.approx(df[k], rel=1e-12, abs=1e-300), k
    for k in ("n_nr", "n_brent", "n_fail", "n_floor", "n_ceil", "n_fixed", "n_steps"):
        assert dr[k] == df[k], k
    if exact_sweeps:
        assert dr["fix_sweeps"] == df["fix_sweeps"]
    assert dr["divb_max"] <= df["divb_max"]


def test_theta_slabs_with_ppm_and_cylindrification():
    """PPM faces (six-zone stencils: all NG = 3 exchanged rows read) on a
    cylindrified grid (each slab's band rows built from their global X2),
    with the failed block across the slab face: bit for bit."""
    kw = dict(recon=O.PPM, cyl_r=1.8, cyl_dx2=0.3)
    state = _torus_start(1, 3, **kw)
    ref = _undecomposed(_base(**kw), state, 2)
    slabs = S.make_theta_slabs(_base(**kw), *state, 3)
    for _ in range(2):
        assert S.step_theta_slabs(slabs)[0] == 0
    P, U, t, dt = S.gather_theta(slabs)
    Pr, Ur, tr, dtr = ref.get_state()
    assert (t, dt) == (tr, dtr)
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)
    assert ref.diagnostics()["n_fixed"] > 0


@pytest.mark.parametrize("R", [2, 3, 4])
def test_theta_slabs_reproduce_the_undecomposed_step(R):
    state = _torus_start(1, R)
    ref = _undecomposed(_base(), state, 3)
    Pr, Ur, tr, dtr = ref.get_state()
    dref = ref.diagnostics()
    assert dref["n_fixed"] >= 70 and dref["fix_sweeps"] >= 5  # the spoiled block, both stages
    slabs = S.make_theta_slabs(_base(), *state, R)
    sweeps = []
    for _ in range(3):
        st, sw = S.step_theta_slabs(slabs)
        assert st == 0
        sweeps += sw
    assert sweeps[0] >= 2 and sweeps[1] >= 2 and sum(sweeps) == dref["fix_sweeps"]
    P, U, t, dt = S.gather_theta(slabs)
    assert t == tr and dt == dtr
    assert np.array_equal(P, Pr)
    assert np.array_equal(U, Ur)
    import torch
    parts = torch.stack([S.oracle_partials(g, 0.0) for g in slabs])
    _check_combined(S.oracle_combine(parts)[0], dref)


def test_theta_slabs_of_a_3d_grid():
    """The same split of a grid with phi zones (the ghost rows carry every
    phi plane and its X3 ghosts)."""
    state = _torus_start(4, 2)
    ref = _undecomposed(_base(4), state, 2)
    slabs = S.make_theta_slabs(_base(4), *state, 2)
    for _ in range(2):
        assert S.step_theta_slabs(slabs)[0] == 0
    P, U, t, dt = S.gather_theta(slabs)
    Pr, Ur, tr, dtr = ref.get_state()
    assert t == tr and dt == dtr and np.array_equal(P, Pr) and np.array_equal(U, Ur)


def _flat_box(n1=12, n2=16, n3=1):
    base = O.default_params(n1=n1, n2=n2, n3=n3, metric=O.MINK_CART, gam=5.0 / 3.0, x1min=0.0, x1max=1.0,
                            x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=O.BC_PERIODIC,
                            bc2=O.BC_PERIODIC, bc3=O.BC_PERIODIC)
    g = O.Grid(base)
    x = (np.arange(n1) + 0.5) / n1
    y = (np.arange(n2) + 0.5) / n2
    X, Y = np.meshgrid(x, y, indexing="ij")
    tp = 2 * np.pi
    P = np.zeros((8, n1, n2, n3))
    P[0] = (1.0 + 0.3 * np.sin(tp * X) * np.cos(tp * Y))[..., None]
    P[1] = (0.6 + 0.2 * np.cos(tp * (X + Y)))[..., None]
    P[2] = (0.3 * np.sin(tp * Y))[..., None]
    P[3] = (-0.2 * np.cos(tp * X))[..., None]
    P[4] = (0.1 * np.sin(tp * (X - Y)))[..., None]
    P[5] = (0.2 + 0.1 * np.sin(tp * Y))[..., None]
    P[6] = (0.1 * np.cos(tp * X))[..., None]
    P[7] = 0.05
    loc = np.repeat(np.arange(n1 * n2, dtype=np.int32), n3)
    U = g.prim2cons(P.reshape(8, -1), loc).reshape((9, n1, n2, n3))
    # spoil a block across the periodic X2 edge: its fixups read across the
    # face that the first and last slabs share
    U = _spoil(U, [n2 - 2, n2 - 1, 0, 1], range(4, 8))
    return base, (P, U, 0.0, 2e-3)


@pytest.mark.parametrize("R", [2, 4])
def test_periodic_theta_slabs_of_a_flat_box(R):
    base, state = _flat_box()
    ref = _undecomposed(base, state, 3)
    slabs = S.make_theta_slabs(base, *state, R, periodic=True)
    for _ in range(3):
        assert S.step_theta_slabs(slabs, periodic=True)[0] == 0
    P, U, t, dt = S.gather_theta(slabs)
    Pr, Ur, tr, dtr = ref.get_state()
    assert ref.diagnostics()["n_fixed"] > 0
    assert t == tr and dt == dtr and np.array_equal(P, Pr) and np.array_equal(U, Ur)


def test_theta_slab_parameters_are_checked():
    with pytest.raises(ValueError):  # fewer than 4 rows
        O.Grid(O.default_params(n1=8, n2=3, n3=1, j0=0, n2_total=6))
    with pytest.raises(ValueError):  # past the whole grid's rows
        O.Grid(O.default_params(n1=8, n2=8, n3=1, j0=4, n2_total=8))
    with pytest.raises(ValueError):  # not also a phi slab
        O.Grid(O.default_params(n1=8, n2=8, n3=4, j0=0, n2_total=16, bc3=O.BC_EXTERNAL))
    g = O.Grid(O.default_params(n1=8, n2=8, n3=1, j0=8, n2_total=16))
    with pytest.raises(RuntimeError):  # a slab takes its state from set_state
        g.init_torus()


def test_theta_slab_geometry_is_the_whole_grids():
    """A slab's metric tables are the whole grid's rows [j0 - NG, j0 + n2 + NG)."""
    whole = O.Grid(_base())
    slab = O.Grid(O.default_params(n1=24, n2=8, n3=1, gam=13.0 / 9.0, r_out=40.0, j0=8, n2_total=24))
    for kind in (0, 1, 2):
        a = whole.geom_table(kind)
        b = slab.geom_table(kind)
        ng = O.NG
        # whole-grid rows j0 - ng .. j0 + n2 + ng of the ghosted table (row index + ng)
        assert np.array_equal(a.reshape(a.shape[0], 24 + 2 * ng, -1)[:, 8:8 + 8 + 2 * ng],
                              b.reshape(b.shape[0], 8 + 2 * ng, -1)), kind


# ---------------------------------------------------- the library's drivers

def test_theta_ring_over_oracle_slabs():
    """ThetaRing (the single-device driver) with the oracle as its engines."""
    from paper_2205_02484_gb300.decomp import ThetaRing
    state = _torus_start(1, 3)
    ref = _undecomposed(_base(), state, 2)
    ring = ThetaRing([S.OracleThetaSlab(S.theta_params(_base(), r, 3)) for r in range(3)])
    assert not ring.device_fix  # oracle engines: the fixup loop runs from the host
    ring.set_state(*state)
    ring.step(1)
    assert ring.sweeps[0] >= 2 and ring.sweeps[1] >= 2  # the block, across the face, both stages
    ring.step(1)
    P = np.concatenate([e.get_state()[0] for e in ring.e], axis=2)
    U = np.concatenate([e.get_state()[1] for e in ring.e], axis=2)
    Pr, Ur, tr, dtr = ref.get_state()
    assert ring.e[0].get_state()[2:] == (tr, dtr)
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)
    _check_combined(ring.diagnostics(), ref.diagnostics())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, steps, periodic, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2205_02484_gb300.decomp import ThetaRank
    from tests import slabs as S2
    from tests import test_oracle_theta_slabs as T
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base, state = T._flat_box() if periodic else (T._base(), T._torus_start(1, world))
    slab = ThetaRank(S2.OracleThetaSlab(S2.theta_params(base, rank, world)), periodic=periodic)
    slab.set_state(*state)
    slab.step(steps)
    P, U, t, dt = slab.e.get_state()
    diag = slab.diagnostics()
    diag["bary"] = slab.barycentric_radius(30.0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (P, U, t, dt, diag))
    dist.destroy_process_group()
    if rank == 0:
        out.put(gathered)


@pytest.mark.parametrize("world,periodic", [(2, False), (3, False), (4, False), (2, True)])
def test_gloo_theta_ranks_reproduce_the_undecomposed_step(world, periodic):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    steps = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, steps, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    base, state = _flat_box() if periodic else (_base(), _torus_start(1, world))
    ref = _undecomposed(base, state, steps)
    Pr, Ur, tr, dtr = ref.get_state()
    P = np.concatenate([g[0] for g in gathered], axis=2)
    U = np.concatenate([g[1] for g in gathered], axis=2)
    assert gathered[0][2] == tr and gathered[0][3] == dtr
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)
    assert all(g[4] == gathered[0][4] for g in gathered)
    _check_combined(gathered[0][4], ref.diagnostics())
    for x, y in zip(gathered[0][4]["bary"], ref.barycentric(30.0)):
        assert x == pytest.approx(y, rel=1e-13, abs=1e-300)


def test_library_theta_grid_parameters():
    """decomp.theta_grid: slab r's rows and the whole grid's, the split's
    checks, and split_theta's parts tiling the whole array."""
    from paper_2205_02484_gb300 import grmhd as G
    from paper_2205_02484_gb300.decomp import split_theta, theta_grid
    base = G.default_grid(24, 48, 1)
    g = theta_grid(base, 4, 3)
    assert (g.n2, g.j0, g.n2_total, g.n1, g.n3) == (12, 36, 48, 24, 1)
    with pytest.raises(ValueError):
        theta_grid(base, 5, 0)   # 48 rows do not split into 5
    with pytest.raises(ValueError):
        theta_grid(base, 16, 0)  # 3-row slabs
    x = np.arange(2 * 24 * 48 * 1, dtype=np.float64).reshape(2, 24, 48, 1)
    parts = [split_theta(x, 4, r) for r in range(4)]
    assert all(p.flags["C_CONTIGUOUS"] for p in parts)
    assert np.array_equal(np.concatenate(parts, axis=2), x)


def _rank_that_leaves(rank, world, port, out):
    """Rank 1 exits after the first exchange (a crash between steps); rank 0's
    next collective of the step must raise instead of waiting forever."""
    import datetime
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2205_02484_gb300.decomp import ThetaRank
    from tests import slabs as S2
    from tests import test_oracle_theta_slabs as T
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    base, state = T._base(), T._torus_start(1, world)
    slab = ThetaRank(S2.OracleThetaSlab(S2.theta_params(base, rank, world)))
    slab.set_state(*state)
    dist.barrier()
    if rank == 1:
        os._exit(0)
    try:
        slab.step(1)
        out.put("no error")
    except Exception as e:  # the process group reports the lost peer
        out.put(f"raised {type(e).__name__}")


def test_a_rank_that_leaves_is_detected():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_that_leaves, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert msg.startswith("raised"), msg
