"""GPU (C ABI) against the oracle: the barycentric radius of Eq. 43 and the
horizon ratio (Edot - Mdot)/|Mdot| on the same torus states, FP64 and mixed;
the empty range; a 4-slab ring's barycentric radius equals the whole grid's."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import gpu_mod, make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _torus_pair(precision, steps=3):
    G = gpu_mod()
    og, ctx = make_pair(48, 32, 8, precision=precision)
    G.init_torus(ctx, pert_amp=0.04, seed=7)
    G.step(ctx, steps)
    P, U, t, dt = G.get_state(ctx)
    og.set_state(P, U, t, dt)
    return G, og, ctx


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("rbar", [12.5, 30.0, 1e9])
def test_barycentric_radius_parity(precision, rbar):
    G, og, ctx = _torus_pair(precision)
    got = G.barycentric_radius(ctx, rbar)
    want = og.barycentric(rbar)
    for x, y in zip(got, want):
        assert x == pytest.approx(y, rel=1e-12)
    assert 6.0 < got[0] < min(rbar, 40.0)


def test_barycentric_radius_empty_range_and_flat_grid():
    G, og, ctx = _torus_pair(0, steps=0)
    assert G.barycentric_radius(ctx, 1.0) == (0.0, 0.0, 0.0)
    gp = G.default_grid(8, 8, 8, metric=G.MINK_CART, x1min=0.0, x1max=1.0, x2min=0.0, x2max=1.0,
                        bc1=G.BC_PERIODIC, bc2=G.BC_PERIODIC)
    flat = G.init_grid(gp, G.default_phys())
    G.set_metric(flat, 0.0, G.MINK_CART)
    P = np.zeros((8, 8, 8, 8))
    P[0], P[1] = 1.0, 0.1
    loc = np.repeat(np.arange(64, dtype=np.int32), 8)
    U = G.prim2cons(flat, P.reshape(8, -1), loc).reshape(9, 8, 8, 8)
    G.set_state(flat, P, U, 0.0, 1e-3)
    with pytest.raises(G.GrmhdError):
        G.barycentric_radius(flat, 10.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_horizon_ratio_parity(precision):
    G, og, ctx = _torus_pair(precision, steps=5)
    dg, do = G.diagnostics(ctx), og.diagnostics()
    assert dg["mdot"] != 0.0
    assert dg["eta"] == pytest.approx(do["eta"], rel=1e-10, abs=1e-14)
    assert dg["eta"] == pytest.approx((dg["edot"] - dg["mdot"]) / abs(dg["mdot"]), rel=1e-15)


def test_slab_ring_barycentric_radius():
    G = gpu_mod()
    from paper_2205_02484_gb300.decomp import SlabRing
    a = 0.9375
    grid = G.default_grid(32, 24, 16, a=a)
    phys = G.default_phys(gam=13.0 / 9.0)
    full = G.init_grid(grid, phys)
    G.set_metric(full, a)
    G.init_torus(full, pert_amp=0.04, seed=3)
    P, U, t, dt = G.get_state(full)
    ring = SlabRing.create(grid, phys, 4, a)
    ring.set_state(P, U, t, dt)
    for x, y in zip(ring.barycentric_radius(30.0), G.barycentric_radius(full, 30.0)):
        assert x == pytest.approx(y, rel=1e-13)
    ring.close()
    full.close()
