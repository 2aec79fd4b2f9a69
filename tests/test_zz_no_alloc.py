"""The allocation-free horizon diagnostics (grmhd_diagnostics_noalloc) give
the same sums as grmhd_diagnostics, on two calls in a row.

Callers that may not allocate device memory (for example an application that
has given all device memory to its own pool) use this entry point; its
reduction scratch is a fixed array inside the library instead of a buffer
allocated with the context.  This file is named so that pytest collects it
last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("mdot", "phib", "edot", "ldot", "divb_max")


def test_noalloc_diagnostics_match_existing_entry_point():
    torch = pytest.importorskip("torch")
    from tests.gpu_common import gpu_mod

    G = gpu_mod()
    gp = G.default_grid(48, 40, 4)
    gp.stream = torch.cuda.current_stream().cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=13.0 / 9.0))
    G.set_metric(ctx, 0.9375, G.KERR_MKS)
    G.init_torus(ctx, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=5)
    G.step(ctx, 3)
    out = torch.full((8,), np.nan, dtype=torch.float64, device="cuda")
    ref = G.diagnostics(ctx)
    for call in range(2):
        G.diagnostics_noalloc(ctx, out)
        G.sync(ctx)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        for idx, key in enumerate(KEYS):
            assert o[idx] == pytest.approx(ref[key], rel=1e-12, abs=1e-300), (call, key, o[idx], ref[key])
        assert np.all(o[5:] == 0.0)
        assert ref["mdot"] != 0.0
    # after further steps the shared array carries the previous call's
    # contents; the next call must not depend on them
    G.step(ctx, 2)
    ref2 = G.diagnostics(ctx)
    G.diagnostics_noalloc(ctx, out)
    G.sync(ctx)
    o = out.cpu().numpy()
    for idx, key in enumerate(KEYS):
        assert o[idx] == pytest.approx(ref2[key], rel=1e-12, abs=1e-300), key
    assert ref2["mdot"] != ref["mdot"]
    ctx.close()


def test_noalloc_rejects_oversized_shell():
    torch = pytest.importorskip("torch")
    from tests.gpu_common import gpu_mod

    G = gpu_mod()
    gp = G.default_grid(2, 2048, 1025, precision=G.MIXED)
    gp.stream = torch.cuda.current_stream().cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=13.0 / 9.0))
    G.set_metric(ctx, 0.9375, G.KERR_MKS)
    P = np.zeros((8, 2, 2048, 1025))
    P[0] = 1.0
    P[1] = 1.0
    U = np.zeros((9, 2, 2048, 1025))
    G.set_state(ctx, P, U, 0.0, 1e-3)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GrmhdError) as e:
        G.diagnostics_noalloc(ctx, out)
    assert e.value.code == -1 and "maximum" in str(e.value)
    ctx.close()
