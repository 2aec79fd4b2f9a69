"""Failure statuses of the C ABI, injected from the host (Sections 2.3-2.4).

* A non-finite value in a state handed to grmhd_set_state is refused with
  GRMHD_ENONFINITE; the context then has no state (grmhd_step: ESTATE) until
  a good state is set.
* A block of zones whose conserved density is negative, wider than the
  fix_maxsweep = 16 Jacobi sweeps of Eq. 33 can fill (each sweep repairs one
  layer from every side), leaves failed zones: grmhd_sync returns
  GRMHD_EFIXUP, like the oracle's step status, the two states still agree,
  and a following grmhd_set_state of a good state steps cleanly.
No kernel faults, traps or waits here: the failures are in the data.
"""
import numpy as np
import pytest

from tests.gpu_common import field_err, gpu_mod, make_pair

pytestmark = pytest.mark.gpu


def _torus(precision=0):
    og, ctx = make_pair(64, 64, 1, gam=13.0 / 9.0, precision=precision)
    og.init_torus(pert_amp=0.04, seed=1)
    return og, ctx, og.get_state()


@pytest.mark.parametrize("where", ["U", "P"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_non_finite_state_is_refused(where, value):
    G = gpu_mod()
    og, ctx, (P, U, t, dt) = _torus()
    Pb, Ub = P.copy(), U.copy()
    (Ub if where == "U" else Pb)[2, 30, 17, 0] = value
    with pytest.raises(G.GrmhdError) as e:
        G.set_state(ctx, Pb, Ub, t, dt)
    assert e.value.code == G.ENONFINITE
    assert "non-finite" in str(e.value)
    with pytest.raises(G.GrmhdError) as e2:
        G.step(ctx)
    assert e2.value.code == G.ESTATE
    # a good state clears it
    G.set_state(ctx, P, U, t, dt)
    G.step(ctx)
    G.sync(ctx)
    og.step()
    assert field_err(G.get_state(ctx)[0], og.get_state()[0]).max() < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_unfixable_block_reports_efixup(precision):
    G = gpu_mod()
    og, ctx, (P, U, t, dt) = _torus(precision)
    Ub = U.copy()
    Ub[0, 14:50, 14:50, :] = -1.0   # 36 x 36 zones: 18 sweeps needed, 16 allowed
    og.set_state(P, Ub, t, dt)
    G.set_state(ctx, P, Ub, t, dt)
    assert og.step() == -1
    G.step(ctx)
    with pytest.raises(G.GrmhdError) as e:
        G.sync(ctx)
    assert e.value.code == G.EFIXUP
    assert "could not be fixed" in str(e.value)
    if precision == 0:
        Po, Uo = og.get_state()[:2]
        Pg, Ug = G.get_state(ctx)[:2]
        assert field_err(Pg, Po).max() < 1e-10
        assert field_err(Ug, Uo).max() < 1e-10
    # the status stays until a new state is set; then the step is clean again
    with pytest.raises(G.GrmhdError):
        G.sync(ctx)
    G.set_state(ctx, P, U, t, dt)
    G.step(ctx, 2)
    G.sync(ctx)
    d = G.diagnostics(ctx)
    assert d["n_steps"] >= 3


def test_fixable_block_is_repaired_within_the_sweep_limit():
    G = gpu_mod()
    og, ctx, (P, U, t, dt) = _torus()
    Ub = U.copy()
    Ub[0, 20:50, 14:44, :] = -1.0   # 30 x 30 zones: 15 sweeps
    og.set_state(P, Ub, t, dt)
    G.set_state(ctx, P, Ub, t, dt)
    assert og.step() == 0
    G.step(ctx)
    G.sync(ctx)
    do, dg = og.diagnostics(), G.diagnostics(ctx)
    assert dg["n_fail"] == do["n_fail"] > 900
    assert dg["fix_sweeps"] == do["fix_sweeps"]
    assert field_err(G.get_state(ctx)[0], og.get_state()[0]).max() < 1e-10
