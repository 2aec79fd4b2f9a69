"""The phi-slab decomposition through the C ABI (grmhd_stage, grmhd_step_dtd,
grmhd_finish_step, grmhd_x3_pack / unpack) on one GPU: R slab contexts
exchanging their X3 ghost planes through device buffers reproduce the
undecomposed GPU step bit for bit, in FP64 and in the mixed path, and the
slab state stays within the per-step parity bound of the undecomposed oracle."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import field_err, gpu_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPE = (32, 24, 16)
GAM = 13.0 / 9.0
A = 0.9375


def _start(G, precision):
    """A perturbed torus (magnetised, so every term of the step is active) as
    host arrays, and an undecomposed context started from it."""
    grid = G.default_grid(*SHAPE, precision=precision, a=A)
    phys = G.default_phys(gam=GAM)
    src = G.init_grid(grid, phys)
    G.set_metric(src, A)
    G.init_torus(src, pert_amp=0.04, seed=11)
    P0, U0, t0, dt0 = G.get_state(src)
    src.close()
    full = G.init_grid(grid, phys)
    G.set_metric(full, A)
    G.set_state(full, P0, U0, t0, dt0)
    return grid, phys, full, (P0, U0, t0, dt0)


def _ring_state(ring):
    parts = [e.get_state() for e in ring.e]
    P = np.concatenate([p[0] for p in parts], axis=3)
    U = np.concatenate([p[1] for p in parts], axis=3)
    return P, U, parts[0][2], parts[0][3]


@pytest.mark.parametrize("precision,R", [(0, 1), (0, 2), (0, 4), (1, 2), (1, 4)])
def test_slab_ring_equals_the_undecomposed_step(precision, R):
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, precision)
    ring = SlabRing.create(grid, phys, R, A)
    ring.set_state(P0, U0, t0, dt0)
    nsteps = 5
    G.step(full, nsteps)
    ring.step(nsteps)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert tr == tf and dtr == dtf
    assert np.array_equal(Pr, Pf)
    assert np.array_equal(Ur, Uf)
    # horizon integrals: the same sums in another order; div B over the
    # corners inside the slabs, a subset of the whole grid's
    df, dr = G.diagnostics(full), ring.diagnostics()
    for k in ("mdot", "phib", "PhiB", "edot", "ldot"):
        assert dr[k] == pytest.approx(df[k], rel=1e-12, abs=1e-300), k
    for k in ("n_nr", "n_fail", "n_floor", "n_fixed"):
        assert dr[k] == df[k], k
    assert dr["divb_max"] <= df["divb_max"]
    ring.close()
    full.close()


@pytest.mark.parametrize("precision,R", [(0, 4), (1, 2)])
def test_slab_ring_with_ppm_and_cylindrification(precision, R):
    """PPM faces (six-zone stencils: all NG = 3 exchanged planes read) on a
    cylindrified grid: the slabs equal the undecomposed step bit for bit."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    grid = G.default_grid(*SHAPE, precision=precision, a=A, recon=G.PPM, cyl_r=1.8, cyl_dx2=0.3)
    phys = G.default_phys(gam=GAM)
    src = G.init_grid(grid, phys)
    G.set_metric(src, A)
    G.init_torus(src, pert_amp=0.04, seed=11)
    P0, U0, t0, dt0 = G.get_state(src)
    src.close()
    full = G.init_grid(grid, phys)
    G.set_metric(full, A)
    G.set_state(full, P0, U0, t0, dt0)
    ring = SlabRing.create(grid, phys, R, A)
    ring.set_state(P0, U0, t0, dt0)
    G.step(full, 3)
    ring.step(3)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert (tr, dtr) == (tf, dtf)
    assert np.array_equal(Pr, Pf) and np.array_equal(Ur, Uf)
    ring.close()
    full.close()


def test_slab_ring_matches_the_oracle_per_step():
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, 0)
    full.close()
    ring = SlabRing.create(grid, phys, 4, A)
    ring.set_state(P0, U0, t0, dt0)
    og = O.Grid(O.default_params(n1=SHAPE[0], n2=SHAPE[1], n3=SHAPE[2], gam=GAM, a=A, r_out=40.0))
    og.set_state(P0, U0, t0, dt0)
    og.step()
    ring.step(1)
    Po, Uo, to, dto = og.get_state()
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert tr == to
    assert dtr == pytest.approx(dto, rel=1e-12)
    assert field_err(Pr, Po).max() < 1e-10
    assert field_err(Ur, Uo).max() < 1e-10
    ring.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_host_launches(precision):
    """A ring step replayed from its CUDA graph equals the same step launched
    kernel by kernel, and a state set after the capture is the one the
    replay steps."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, precision)
    full.close()
    a = SlabRing.create(grid, phys, 4, A)
    b = SlabRing.create(grid, phys, 4, A)
    a.set_state(P0, U0, t0, dt0)
    b.set_state(P0, U0, t0, dt0)
    a.step(3, graph=False)
    b.step(3)
    assert b._graph is not None
    Pa, Ua, ta, dta = _ring_state(a)
    Pb, Ub, tb, dtb = _ring_state(b)
    assert (ta, dta) == (tb, dtb)
    assert np.array_equal(Pa, Pb) and np.array_equal(Ua, Ub)
    b.set_state(P0, U0, t0, dt0)
    b.step(3)
    Pc, Uc, tc, dtc = _ring_state(b)
    assert (tc, dtc) == (ta, dta)
    assert np.array_equal(Pc, Pa) and np.array_equal(Uc, Ua)
    a.close()
    b.close()


def test_pack_unpack_planes():
    """pack copies the two outermost active planes of a side; unpack writes
    the ghost planes the step reads (checked through a one-slab ring, whose
    ghosts are its own opposite planes, against the periodic fill)."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    grid, phys, full, (P0, U0, t0, dt0) = _start(G, 0)
    full.close()
    ring = SlabRing.create(grid, phys, 1, A)
    ring.set_state(P0, U0, t0, dt0)
    e = ring.e[0]
    buf = torch.empty(e.plane_numel, dtype=torch.float64, device="cuda")
    ng = G.NG
    for side, ks in ((0, tuple(range(ng))), (1, tuple(range(SHAPE[2] - ng, SHAPE[2])))):
        e.pack(0, side, buf)
        torch.cuda.synchronize()
        planes = buf.cpu().numpy().reshape(ng, 8, SHAPE[0] + 2 * ng, SHAPE[1] + 2 * ng)
        for g, k in enumerate(ks):
            # the active part of the packed plane is the state's plane k
            assert np.array_equal(planes[g, :, G.NG:-G.NG, G.NG:-G.NG], P0[:, :, :, k])
    assert G.x3_plane_bytes(e.ctx) == ng * 8 * (SHAPE[0] + 2 * ng) * (SHAPE[1] + 2 * ng) * 8
    with pytest.raises(G.GrmhdError):
        G.x3_pack(e.ctx, 2, 0, buf)
    with pytest.raises(G.GrmhdError):
        G.x3_unpack(e.ctx, 0, -1, buf)
    with pytest.raises(G.GrmhdError):
        G.stage(e.ctx, 3)
    with pytest.raises(G.GrmhdError):  # a slab steps stage by stage, with exchanges
        G.step(e.ctx, 1)
    ring.close()


def test_external_is_for_bc3_only():
    G = gpu_mod()
    with pytest.raises(G.GrmhdError):
        G.init_grid(G.default_grid(8, 8, 8, bc1=G.BC_EXTERNAL), G.default_phys())
    with pytest.raises(G.GrmhdError):
        G.init_grid(G.default_grid(8, 8, 1, bc3=G.BC_EXTERNAL), G.default_phys())


@pytest.mark.parametrize("precision,R", [(0, 2), (1, 4)])
def test_flat_space_slabs_equal_the_undecomposed_step(precision, R):
    """The phi (X3) split of a flat-space periodic box: a smooth MHD state
    stepped as R slabs equals the undecomposed box bit for bit (the slab X3
    ranges [0, (n3 / R) dX3) keep dX3 exact for power-of-two widths)."""
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    n1, n2, n3 = 12, 10, 16
    grid = G.default_grid(n1, n2, n3, metric=G.MINK_CART, precision=precision, x1min=0.0, x1max=1.0,
                          x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=G.BC_PERIODIC, bc2=G.BC_PERIODIC,
                          bc3=G.BC_PERIODIC)
    phys = G.default_phys(gam=5.0 / 3.0)
    full = G.init_grid(grid, phys)
    G.set_metric(full, 0.0, G.MINK_CART)
    x = (np.arange(n1) + 0.5) / n1
    y = (np.arange(n2) + 0.5) / n2
    z = (np.arange(n3) + 0.5) / n3
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    tp = 2 * np.pi
    P = np.zeros((8, n1, n2, n3))
    P[0] = 1.0 + 0.3 * np.sin(tp * X) * np.cos(tp * Z)
    P[1] = 0.6 + 0.2 * np.cos(tp * (Y + Z))
    P[2] = 0.3 * np.sin(tp * Z)
    P[3] = -0.2 * np.cos(tp * X)
    P[4] = 0.25 * np.sin(tp * (X - Z))
    P[5] = 0.2 + 0.1 * np.sin(tp * Y)
    P[6] = 0.1 * np.cos(tp * Z)
    P[7] = 0.15 * np.sin(tp * X)
    loc = np.zeros(n1 * n2 * n3, dtype=np.int32)
    U = G.prim2cons(full, P.reshape(8, -1), loc).reshape((9, n1, n2, n3))
    dt = 2e-3
    G.set_state(full, P, U, 0.0, dt)
    ring = SlabRing.create(grid, phys, R, 0.0)
    ring.set_state(P, U, 0.0, dt)
    G.step(full, 4)
    ring.step(4)
    Pf, Uf, tf, dtf = G.get_state(full)
    Pr, Ur, tr, dtr = _ring_state(ring)
    assert tr == tf and dtr == dtf
    assert np.array_equal(Pr, Pf) and np.array_equal(Ur, Uf)
    ring.close()
    full.close()
