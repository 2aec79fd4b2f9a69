"""grmhd_set_state_u: a state given by its conserved variables alone, the
primitives re-derived on the device by the step's inversion, floors and
fixups (Sections 2.3-2.4, Eq. 33).

* After a step P is the inversion of U, so a context handed back the U that
  grmhd_get_state returned recovers the primitives to the inversion's
  tolerance and steps on as the context that kept its full state (FP64 path:
  1e-10 per field, the metric of gpu_common.field_err; mixed path: the
  mixed inversion's 1e-4), host and device U alike.
* Starting Newton from older primitives (a context a few steps behind)
  reaches the same primitives.
* The oracle, stepping the full state, agrees with a step taken after
  set_state_u as with any step.
* Refusals: no state to start from, a non-finite U, a slab, bad t / dt.
"""
import numpy as np
import pytest
import torch

from tests.gpu_common import field_err, gpu_mod, make_pair

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _pair(precision=0, n3=1):
    og, ctx = make_pair(64, 64, n3, gam=13.0 / 9.0, precision=precision)
    og.init_torus(pert_amp=0.04, seed=1)
    return og, ctx


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("device", [False, True])
def test_round_trip_of_the_conserved_state(precision, device):
    G = gpu_mod()
    og, a = _pair(precision)
    _, b = _pair(precision)
    G.init_torus(a, pert_amp=0.04, seed=1)
    G.step(a, 3)
    Pa, Ua, ta, dta = G.get_state(a)
    G.set_state(b, Pa, Ua, ta, dta)
    if device:
        Ud = torch.from_numpy(Ua).cuda()
        G.set_state_u(b, Ud, ta, dta)
        Uh = torch.empty_like(Ud)
        Uh, tb, dtb = G.get_state_u(b, Uh)
        Ub = Uh.cpu().numpy()
    else:
        G.set_state_u(b, Ua, ta, dta)
        Ub, tb, dtb = G.get_state_u(b)
    Pb = G.get_state(b)[0]
    assert tb == ta and dtb == dta
    # U passes through (a zone re-floored by rounding has its U recomputed
    # from its primitives: U_S, the entropy, then moves by the inversion's
    # tolerance; on the mixed path by the FP32 rounding); P comes back to the
    # inversion's tolerance (FP64), or the mixed inversion's (Newton accepted
    # at a step below sqrt(nr_tol); u of cold gas carries ~rho/u times that)
    tolP = 1e-9 if precision == 0 else 1e-4
    eU = field_err(Ub, Ua)
    if precision == 0:
        assert eU[:8].max() < 1e-14 and eU[8] < TOL, eU
    else:
        assert eU.max() < 1e-6, eU
    assert field_err(Pb, Pa).max() < tolP, field_err(Pb, Pa)
    G.step(a, 2)
    G.step(b, 2)
    tol = TOL if precision == 0 else 1e-4
    assert field_err(G.get_state(b)[0], G.get_state(a)[0]).max() < tol
    assert field_err(G.get_state(b)[1], G.get_state(a)[1]).max() < tol
    G.sync(b)


def test_newton_from_older_primitives():
    G = gpu_mod()
    og, a = _pair()
    _, b = _pair()
    G.init_torus(a, pert_amp=0.04, seed=1)
    G.init_torus(b, pert_amp=0.04, seed=1)
    G.step(a, 4)
    Pa, Ua, ta, dta = G.get_state(a)
    d0 = G.diagnostics(b)
    G.set_state_u(b, Ua, ta, dta)        # b still holds the initial primitives
    d1 = G.diagnostics(b)
    Pb = G.get_state(b)[0]
    assert field_err(Pb, Pa).max() < 1e-9, field_err(Pb, Pa)
    inversions = sum(d1[k] - d0[k] for k in ("n_nr", "n_brent", "n_entropy", "n_entropy_beta", "n_fail"))
    assert inversions == 64 * 64


def test_step_after_set_state_u_matches_the_oracle():
    G = gpu_mod()
    og, ctx = _pair()
    Po, Uo, to, dto = og.get_state()
    G.set_state(ctx, Po, Uo, to, dto)
    for _ in range(3):
        og.step()
        Po, Uo, to, dto = og.get_state()
        G.set_state_u(ctx, Uo, to, dto)   # the oracle's U; the GPU's own P as the start
        og.step()
        G.step(ctx)
        eP = field_err(G.get_state(ctx)[0], og.get_state()[0])
        eU = field_err(G.get_state(ctx)[1], og.get_state()[1])
        assert max(eP.max(), eU.max()) < TOL, (eP, eU)


def test_refusals():
    G = gpu_mod()
    og, ctx = _pair()
    U = og.get_state()[1]
    with pytest.raises(G.GrmhdError) as e:
        G.set_state_u(ctx, U, 0.0, 1e-3)     # nothing to start Newton from
    assert e.value.code == G.ESTATE
    Po, Uo, to, dto = og.get_state()
    G.set_state(ctx, Po, Uo, to, dto)
    for t, dt in ((np.nan, 1e-3), (0.0, np.inf), (0.0, -1.0)):
        with pytest.raises(G.GrmhdError) as e:
            G.set_state_u(ctx, Uo, t, dt)
        assert e.value.code == G.EINVAL
    bad = Uo.copy()
    bad[2, 5, 7, 0] = np.nan
    with pytest.raises(G.GrmhdError) as e:
        G.set_state_u(ctx, bad, to, dto)
    assert e.value.code == G.ENONFINITE
    with pytest.raises(G.GrmhdError):
        G.step(ctx)                           # no state until a good one is set
    G.set_state(ctx, Po, Uo, to, dto)
    G.set_state_u(ctx, Uo, to, dto)
    G.step(ctx)
    G.sync(ctx)
