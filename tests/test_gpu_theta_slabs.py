"""The theta-slab decomposition through the C ABI (grmhd_stage_update,
grmhd_fail_count, grmhd_fix_sweep, grmhd_fix_end, grmhd_stage_bc,
grmhd_x2_pack / unpack, and grmhd_theta_ring_fix, the same fixup loop on the
device) on one GPU: R slab contexts exchanging their X2 ghost rows, and
before every fixup sweep the edge rows a sweep reads across a slab face,
reproduce the undecomposed GPU step bit for bit in FP64 and in the mixed
path, with the fixup loop run from the host or on the device, stepped kernel
by kernel or replayed from a CUDA graph; the slab state stays within the
per-step parity bound of the undecomposed oracle.  A block of zones made to
fail (negative conserved density) straddles a slab face, so the fixups of
Eq. 33 run several sweeps across it in both stages."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import field_err, gpu_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAM = 13.0 / 9.0
A = 0.9375


def _spoil(U, rows, cols):
    U = U.copy()
    for j in rows:
        for i in cols:
            U[0, i, j, :] = -1.0
    return U


def _start(G, precision, R, shape=(40, 48, 1), riemann=0, **kw):
    grid = G.default_grid(*shape, precision=precision, a=A, riemann=riemann, **kw)
    phys = G.default_phys(gam=GAM)
    src = G.init_grid(grid, phys)
    G.set_metric(src, A)
    G.init_torus(src, pert_amp=0.04, seed=11)
    P0, U0, t0, dt0 = G.get_state(src)
    src.close()
    b = shape[1] // R  # the first inner slab face
    c0 = min(14, shape[0] - 8)
    U0 = _spoil(U0, range(b - 3, b + 3), range(c0, c0 + 7))
    full = G.init_grid(grid, phys)
    G.set_metric(full, A)
    G.set_state(full, P0, U0, t0, dt0)
    return grid, phys, full, (P0, U0, t0, dt0)


def _ring_state(ring):
    parts = [e.get_state() for e in ring.e]
    P = np.concatenate([p[0] for p in parts], axis=2)
    U = np.concatenate([p[1] for p in parts], axis=2)
    return P, U, parts[0][2], parts[0][3]


@pytest.mark.parametrize("precision,R,riemann,device_fix,graph",
                         [(0, 2, 0, True, True), (0, 3, 0, True, True), (0, 4, 0, True, True),
                          (1, 2, 0, True, True), (1, 4, 0, True, True), (1, 3, 1, True, True),
                          (0, 4, 0, False, False), (1, 3, 1, False, False), (0, 3, 0, True, False)])
def test_theta_ring_equals_the_undecomposed_step(precision, R, riemann, device_fix, graph):
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, precision, R, riemann=riemann)
    ring = ThetaRing.create(grid, phys, R, A, device_fix=device_fix)
    assert ring.device_fix == device_fix
    ring.set_state(P0, U0, t0, dt0)
    nsteps = 4
    G.step(full, 1)
    ring.step(1, graph=graph)
    assert ring.sweeps[0] >= 2 and ring.sweeps[1] >= 2  # the block, across the face, both stages
    G.step(full, nsteps - 1)
    ring.step(nsteps - 1, graph=graph)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert tr == tf and dtr == dtf
    assert np.array_equal(Pr, Pf)
    assert np.array_equal(Ur, Uf)
    df, dr = G.diagnostics(full), ring.diagnostics()
    for k in ("mdot", "phib", "PhiB", "edot", "ldot"):
        assert dr[k] == pytest.approx(df[k], rel=1e-12, abs=1e-300), k
    for k in ("n_nr", "n_fail", "n_floor", "n_fixed", "fix_sweeps", "n_steps"):
        assert dr[k] == df[k], k
    assert df["n_fixed"] >= 70
    assert dr["divb_max"] <= df["divb_max"]
    ring.close()
    full.close()


@pytest.mark.parametrize("precision,R", [(0, 3), (1, 4)])
def test_theta_ring_with_ppm_and_cylindrification(precision, R):
    """PPM faces (six-zone stencils: all NG = 3 exchanged rows read) on a
    cylindrified grid (the band rows' metric built from their global X2
    positions in every slab), with the failed block across a slab face:
    the ring equals the undecomposed step bit for bit."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, precision, R, recon=G.PPM, cyl_r=1.8, cyl_dx2=0.3)
    ring = ThetaRing.create(grid, phys, R, A)
    ring.set_state(P0, U0, t0, dt0)
    G.step(full, 3)
    ring.step(3)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert (tr, dtr) == (tf, dtf)
    assert np.array_equal(Pr, Pf) and np.array_equal(Ur, Uf)
    df, dr = G.diagnostics(full), ring.diagnostics()
    assert df["n_fixed"] > 0
    for k in ("n_nr", "n_fail", "n_floor", "n_fixed", "fix_sweeps"):
        assert dr[k] == df[k], k
    ring.close()
    full.close()


def test_theta_ring_matches_the_oracle_per_step():
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    shape = (40, 48, 1)
    grid, phys, full, state = _start(G, 0, 4, shape)
    full.close()
    ring = ThetaRing.create(grid, phys, 4, A)
    ring.set_state(*state)
    og = O.Grid(O.default_params(n1=shape[0], n2=shape[1], n3=shape[2], gam=GAM, a=A, r_out=40.0))
    og.set_state(*state)
    assert og.step() == 0
    ring.step(1)
    Po, Uo, to, dto = og.get_state()
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert tr == to
    assert dtr == pytest.approx(dto, rel=1e-12)
    assert field_err(Pr, Po).max() < 1e-10
    assert field_err(Ur, Uo).max() < 1e-10
    assert ring.diagnostics()["n_fixed"] == og.diagnostics()["n_fixed"]
    ring.close()


def test_theta_slabs_of_a_3d_grid():
    """The theta split of a grid with phi zones: the ghost rows carry every
    phi plane with its X3 ghosts."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    grid, phys, full, state = _start(G, 0, 2, (24, 16, 8))
    ring = ThetaRing.create(grid, phys, 2, A)
    ring.set_state(*state)
    G.step(full, 3)
    ring.step(3)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert (tr, dtr) == (tf, dtf)
    assert np.array_equal(Pr, Pf) and np.array_equal(Ur, Uf)
    ring.close()
    full.close()


@pytest.mark.parametrize("precision,device_fix", [(0, True), (1, True), (0, False)])
def test_periodic_flat_box_theta_slabs(precision, device_fix):
    """A flat periodic box split in X2: the first and last slabs are
    neighbours, and a failed block across the periodic edge is fixed from
    both sides."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    n1, n2, n3 = 12, 16, 1
    grid = G.default_grid(n1, n2, n3, metric=G.MINK_CART, precision=precision, x1min=0.0, x1max=1.0,
                          x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=G.BC_PERIODIC, bc2=G.BC_PERIODIC,
                          bc3=G.BC_PERIODIC)
    phys = G.default_phys(gam=5.0 / 3.0)
    full = G.init_grid(grid, phys)
    G.set_metric(full, 0.0, G.MINK_CART)
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
    loc = np.zeros(n1 * n2 * n3, dtype=np.int32)
    U = G.prim2cons(full, P.reshape(8, -1), loc).reshape((9, n1, n2, n3))
    U = _spoil(U, [n2 - 2, n2 - 1, 0, 1], range(4, 8))
    dt = 2e-3
    G.set_state(full, P, U, 0.0, dt)
    ring = ThetaRing.create(grid, phys, 2, 0.0, periodic=True, device_fix=device_fix)
    ring.set_state(P, U, 0.0, dt)
    G.step(full, 3)
    ring.step(3)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert (tr, dtr) == (tf, dtf)
    assert np.array_equal(Pr, Pf) and np.array_equal(Ur, Uf)
    assert G.diagnostics(full)["n_fixed"] > 0
    ring.close()
    full.close()


def test_theta_pack_unpack_rows_and_errors():
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    shape = (20, 16, 1)
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, 0, 2, shape)
    full.close()
    ring = ThetaRing.create(grid, phys, 2, A)
    ring.set_state(P0, U0, t0, dt0)
    e0, e1 = ring.e
    n1, n2, n3 = shape[0], shape[1] // 2, shape[2]
    ng = G.NG
    assert G.x2_row_bytes(e0.ctx, 0) == ng * 8 * (n1 + 2 * ng) * (n3 + 2 * ng) * 8
    assert G.x2_row_bytes(e0.ctx, 1) == 6 * n1 * n3 * 8
    buf = torch.empty(e0.row_numel, dtype=torch.float64, device="cuda")
    for side, js in ((0, tuple(range(ng))), (1, tuple(range(n2 - ng, n2)))):
        e0.pack(0, 0, side, buf)
        torch.cuda.synchronize()
        rows = buf.cpu().numpy().reshape(ng, 8, n1 + 2 * ng, n3 + 2 * ng)
        for g, j in enumerate(js):
            assert np.array_equal(rows[g, :, ng:-ng, ng:-ng], P0[:, :, j, :])
    fb = torch.empty(e0.fix_numel, dtype=torch.float64, device="cuda")
    e1.pack(1, 0, 0, fb)
    torch.cuda.synchronize()
    rows = fb.cpu().numpy().reshape(6, n1, n3)
    assert np.array_equal(rows[:5], P0[:5, :, n2, :])
    assert set(np.unique(rows[5])) <= {0.0, 1.0}
    # the ghost rows after set_state hold the neighbour's edge rows
    e1.unpack(0, 0, 0, buf)  # (no-op check of the call on a slab)
    with pytest.raises(ValueError):  # a short buffer
        G.x2_pack(e0.ctx, 0, 0, 0, fb)
    with pytest.raises(G.GrmhdError):
        G.x2_pack(e0.ctx, 2, 0, 0, buf)
    with pytest.raises(G.GrmhdError):
        G.x2_unpack(e0.ctx, 0, 0, -1, buf)
    with pytest.raises(G.GrmhdError):  # a theta slab steps by the stage parts
        G.step(e0.ctx, 1)
    with pytest.raises(G.GrmhdError):
        G.stage(e0.ctx, 0)
    with pytest.raises(G.GrmhdError):  # its state comes from set_state
        G.init_torus(e0.ctx)
    with pytest.raises(G.GrmhdError):  # a slab is not an ensemble member
        G.ensemble_create([e0.ctx])
    whole = G.init_grid(G.default_grid(*shape, a=A), phys)
    G.set_metric(whole, A)
    G.set_state(whole, P0, U0, t0, dt0)
    with pytest.raises(G.GrmhdError):  # the parts are for theta slabs
        G.stage_update(whole, 0)
    with pytest.raises(G.GrmhdError):
        G.x2_pack(whole, 0, 0, 0, buf)
    whole.close()
    ring.close()


def test_graph_replay_after_set_state():
    """A state set after the ring's graph was captured is the one replayed:
    the same steps from the same start give the same bits and sweep counts."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    grid, phys, full, state = _start(G, 1, 4)
    full.close()
    ring = ThetaRing.create(grid, phys, 4, A)
    ring.set_state(*state)
    ring.step(2)
    P1, U1, t1, dt1 = _ring_state(ring)
    sw1 = ring.sweeps
    ring.set_state(*state)
    ring.step(2)
    P2, U2, t2, dt2 = _ring_state(ring)
    assert (t1, dt1) == (t2, dt2) and ring.sweeps == sw1
    assert np.array_equal(P1, P2) and np.array_equal(U1, U2)
    ring.close()


def test_sixteen_slab_ring_and_the_limit():
    """16 slabs of 4 rows (the most one ring kernel takes: their grid records
    travel as one parameter block) equal the undecomposed step, failed block
    included; 17 are refused by grmhd_theta_ring_fix."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    grid, phys, full, state = _start(G, 0, 16, shape=(24, 64, 1))
    ring = ThetaRing.create(grid, phys, 16, A)
    ring.set_state(*state)
    G.step(full, 2)
    ring.step(2)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert (tr, dtr) == (tf, dtf)
    assert np.array_equal(Pr, Pf) and np.array_equal(Ur, Uf)
    assert G.diagnostics(full)["n_fixed"] > 0
    nsw = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GrmhdError) as e:
        G.theta_ring_fix([e_.ctx for e_ in ring.e] + [ring.e[0].ctx], 0, nsw)
    assert e.value.code == G.EINVAL
    ring.close()
    full.close()


def test_ring_fix_refusals():
    """grmhd_theta_ring_fix takes the slabs of one grid, in theta order,
    covering every row, on one stream; a refusal launches nothing."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import ThetaRing
    grid, phys, full, state = _start(G, 0, 4)
    full.close()
    ring = ThetaRing.create(grid, phys, 4, A)
    ring.set_state(*state)
    c = [e.ctx for e in ring.e]
    nsw = torch.zeros(1, dtype=torch.int32, device="cuda")
    for bad in (c[1:], c[:3], [c[0], c[2], c[1], c[3]], [c[0], c[0], c[2], c[3]]):
        with pytest.raises(G.GrmhdError) as e:
            G.theta_ring_fix(bad, 0, nsw)
        assert e.value.code == G.EINVAL
    with pytest.raises(G.GrmhdError):
        G.theta_ring_fix(c, 2, nsw)
    other = ThetaRing.create(grid, phys, 4, A)     # its own stream
    other.set_state(*state)
    with pytest.raises(G.GrmhdError):
        G.theta_ring_fix([c[0], c[1], other.e[2].ctx, c[3]], 0, nsw)
    with pytest.raises(ValueError):
        G.theta_ring_fix(c, 0, torch.zeros(1, dtype=torch.int64, device="cuda"))
    G.theta_ring_fix(c, 0, nsw)                    # nothing failed before a stage: no sweep
    assert int(nsw.cpu()[0]) == 0
    other.close()
    ring.close()


def test_theta_slab_parameters_are_checked():
    G = gpu_mod()
    phys = G.default_phys()
    for kw in (dict(n2=3, j0=0, n2_total=6), dict(n2=8, j0=4, n2_total=8), dict(n2=8, j0=2, n2_total=0),
               dict(n2=8, j0=0, n2_total=16, n3=4, bc3=G.BC_EXTERNAL)):
        n3 = kw.pop("n3", 1)
        with pytest.raises(G.GrmhdError):
            G.init_grid(G.default_grid(8, kw.pop("n2"), n3, **kw), phys)
