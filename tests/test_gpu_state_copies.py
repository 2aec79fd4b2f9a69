"""Host <-> device state copies through the C ABI (grmhd_set_state /
grmhd_get_state): a state large enough that the copy is split into several
byte ranges on several streams, with a range crossing from P into U, comes
back bit for bit through host buffers, equals the same state passed as
device tensors, and steps identically; P alone or U alone is copied too."""
import numpy as np
import pytest

from tests.gpu_common import gpu_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_split_host_copies_round_trip_and_step():
    G = gpu_mod()
    shape = (64, 64, 32)  # 17.8 MB of P and U: four ranges of 5 MiB
    grid = G.default_grid(*shape, a=0.9375)
    phys = G.default_phys()
    src = G.init_grid(grid, phys)
    G.set_metric(src, 0.9375)
    G.init_torus(src, pert_amp=0.04, seed=21)
    P0, U0, t0, dt0 = G.get_state(src)
    src.close()
    # pinned and pageable host buffers, and device tensors
    Pp = torch.from_numpy(P0).pin_memory()
    Up = torch.from_numpy(U0).pin_memory()
    a, b = G.init_grid(grid, phys), G.init_grid(grid, phys)
    for c in (a, b):
        G.set_metric(c, 0.9375)
    G.set_state(a, Pp.numpy(), Up.numpy(), t0, dt0)
    G.set_state(b, Pp.cuda(), Up.cuda(), t0, dt0)
    Pa, Ua, ta, dta = G.get_state(a)
    assert np.array_equal(Pa, P0) and np.array_equal(Ua, U0) and (ta, dta) == (t0, dt0)
    Pd = torch.empty_like(Pp, device="cuda")
    Ud = torch.empty_like(Up, device="cuda")
    G.get_state(b, Pd, Ud)
    assert np.array_equal(Pd.cpu().numpy(), P0) and np.array_equal(Ud.cpu().numpy(), U0)
    G.step(a, 2)
    G.step(b, 2)
    Pa, Ua, _, _ = G.get_state(a)
    Pb, Ub, _, _ = G.get_state(b)
    assert np.array_equal(Pa, Pb) and np.array_equal(Ua, Ub)
    # one part alone (its own ranges; the other pointer NULL) into pinned buffers
    Ponly = torch.zeros_like(Pp).pin_memory().numpy()
    Uonly = torch.zeros_like(Up).pin_memory().numpy()
    assert a.L.grmhd_get_state(a.h, Ponly.ctypes.data, None, None, None, 0) == 0
    assert a.L.grmhd_get_state(a.h, None, Uonly.ctypes.data, None, None, 0) == 0
    assert np.array_equal(Ponly, Pa) and np.array_equal(Uonly, Ua)
    a.close()
    b.close()
