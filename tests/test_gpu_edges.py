"""Edge cases of the C ABI and of the step on the GPU: empty and ragged
batches (warps and blocks partly filled, the tensor-core inference's lanes
past the batch), zone locations outside the grid, grid-size limits, and
grids down to one zone per direction (every stencil then reads ghosts that
the boundary fill made from the same few zones), against the oracle."""
import numpy as np
import pytest

import oracle
from tests import inputs
from tests.gpu_common import field_err, gpu_mod, make_pair
from tests.michel import Michel, michel_prims

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _states(og, n, seed, n1, n2):
    tab = og.geom_table(0)
    loc = inputs.zone_locations(n, n1, n2, seed, i_h=og.i_h)
    i, j = loc // n2, loc % n2
    gsp = tab[i + oracle.NG, j + oracle.NG, :16].reshape(n, 4, 4)[:, 1:, 1:]
    P = inputs.place_prims(inputs.prim_params(n, seed + 1), gsp)
    return loc, P, og.prim2cons(P, loc)


def test_empty_batches():
    G = gpu_mod()
    og, ctx = make_pair(16, 16, 1, gam=4.0 / 3.0)
    U = np.zeros((9, 0))
    P = np.zeros((8, 0))
    loc = np.zeros(0, dtype=np.int32)
    Pg, fl, it = G.con2prim(ctx, U, loc, P)
    assert Pg.shape == (8, 0) and fl.shape == (0,) and it.shape == (0,)
    assert G.prim2cons(ctx, P, loc).shape == (9, 0)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ragged_batches_equal_the_full_batch(mode):
    """The first n states of a 256-state batch, inverted alone, give the
    full batch's answers: n = 1 (one lane of one warp), 31, 33 (a warp and
    one lane), 129 (a block and one lane)."""
    G = gpu_mod()
    n1, n2 = 24, 20
    og, ctx = make_pair(n1, n2, 1, gam=4.0 / 3.0, r_out=1000.0)
    loc, P, U = _states(og, 256, 41, n1, n2)
    if mode:
        rng = np.random.default_rng(3)
        th = (0.05 * rng.standard_normal(oracle.MLP_NPARAM)).astype(np.float32)
        nm = np.array([0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 0, 1], dtype=np.float32)
        G.mlp_load(ctx, th, nm)
    guess = P * (1.0 + 1e-4 * np.sin(np.arange(P.size)).reshape(P.shape))
    guess[5:8] = P[5:8]
    Pf, ff, itf = G.con2prim(ctx, U, loc, guess.copy(), use_learned_guess=mode)
    for n in (1, 31, 33, 129):
        Pn, fn, itn = G.con2prim(ctx, np.ascontiguousarray(U[:, :n]), loc[:n].copy(),
                                 np.ascontiguousarray(guess[:, :n]), use_learned_guess=mode)
        assert np.array_equal(fn, ff[:n]), n
        assert np.array_equal(itn, itf[:n]), n
        assert np.array_equal(Pn, Pf[:, :n]), n
    # prim2cons of a ragged batch: the full batch's values (its parity with the
    # oracle is tested in test_gpu_parity)
    Ufull = G.prim2cons(ctx, P, loc)
    assert np.array_equal(G.prim2cons(ctx, np.ascontiguousarray(P[:, :33]), loc[:33].copy()), Ufull[:, :33])


def test_locations_outside_the_grid_fail_alone():
    G = gpu_mod()
    n1, n2 = 16, 12
    og, ctx = make_pair(n1, n2, 1, gam=4.0 / 3.0)
    loc, P, U = _states(og, 64, 7, n1, n2)
    bad = loc.copy()
    bad[[3, 40]] = [-1, n1 * n2]
    Pa, fa, _ = G.con2prim(ctx, U, loc, P.copy())
    Pb, fb, _ = G.con2prim(ctx, U, bad, P.copy())
    assert fb[3] == fb[40] == G.C2P_FAIL | G.C2P_FAIL_D
    keep = np.setdiff1d(np.arange(64), [3, 40])
    assert np.array_equal(fb[keep], fa[keep])
    assert np.array_equal(Pb[:, keep], Pa[:, keep])


@pytest.mark.parametrize("dims,kerr", [((1290, 1290, 1290), False), ((0, 8, 8), False), ((8, 8, 0), False),
                                       ((1, 8, 8), True)])
def test_grid_size_limits(dims, kerr):
    """More than 2^31 - 1 zones with ghosts (the zone lists are 32-bit), an
    empty direction, and a Kerr grid of one radial zone are refused before
    any allocation."""
    G = gpu_mod()
    kw = {} if kerr else dict(metric=G.MINK_CART)
    gp = G.default_grid(*dims, **kw)
    with pytest.raises(G.GrmhdError) as e:
        G.init_grid(gp, G.default_phys())
    assert e.value.code == G.EINVAL


@pytest.mark.parametrize("recon", [oracle.PLM, oracle.PPM])
def test_smallest_kerr_grid(recon):
    """4 x 6 x 2 zones of Michel's flow on a = 0 (six rows: the polar
    interpolation of two rows per pole from the third), two steps per step."""
    G = gpu_mod()
    og, ctx = make_pair(4, 6, 2, gam=4.0 / 3.0, a=0.0, r_out=20.0, recon=recon)
    P = michel_prims(og, Michel(r_c=8.0, n=3.0), 4.0 / 3.0)
    loc = np.repeat((np.arange(4)[:, None] * 6 + np.arange(6)[None, :]).reshape(-1), 2).astype(np.int32)
    U = og.prim2cons(P.reshape(8, -1), loc).reshape((9,) + og.shape)
    og.set_state(P, U, 0.0, 0.0)
    dt = og.initial_dt()
    og.set_state(P, U, 0.0, dt)
    for _ in range(2):
        Po, Uo, to, dto = og.get_state()
        G.set_state(ctx, Po, Uo, to, dto)
        og.step()
        G.step(ctx)
        eP = field_err(G.get_state(ctx)[0], og.get_state()[0])
        eU = field_err(G.get_state(ctx)[1], og.get_state()[1])
        assert max(eP.max(), eU.max()) < TOL, (eP, eU)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3), (3, 2, 1)])
@pytest.mark.parametrize("recon", [oracle.PLM, oracle.PPM])
def test_one_zone_periodic_boxes(shape, recon):
    """Flat periodic boxes down to one zone: every face reads ghosts that are
    copies of the same zones, so the state must stay exactly uniform along a
    direction of one zone; against the oracle per field."""
    G = gpu_mod()
    n1, n2, n3 = shape
    box = dict(x1min=0.0, x1max=1.0, x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=oracle.BC_PERIODIC,
               bc2=oracle.BC_PERIODIC, bc3=oracle.BC_PERIODIC, recon=recon)
    og, ctx = make_pair(n1, n2, n3, gam=5.0 / 3.0, metric=oracle.MINK_CART, **box)
    rng = np.random.default_rng(5)
    P = np.zeros((8, n1, n2, n3))
    P[0] = 1.0 + 0.2 * rng.random(shape)
    P[1] = 0.5 + 0.1 * rng.random(shape)
    P[2:5] = 0.2 * (rng.random((3,) + shape) - 0.5)
    P[5:8] = 0.1                       # uniform field: divergence free on any box
    U = og.prim2cons(P.reshape(8, -1), np.repeat(np.arange(n1 * n2, dtype=np.int32), n3)).reshape((9,) + shape)
    og.set_state(P, U, 0.0, 0.0)
    dt = og.initial_dt()
    og.set_state(P, U, 0.0, dt)
    G.set_state(ctx, P, U, 0.0, dt)
    for _ in range(2):
        og.step()
        G.step(ctx)
    Pg, Po = G.get_state(ctx)[0], og.get_state()[0]
    assert field_err(Pg, Po).max() < 1e-9
    # a single zone in every direction: nothing changes at all
    if shape == (1, 1, 1):
        assert np.abs(Pg - P).max() < 1e-13 * np.abs(P).max()
