"""Parity at the benchmark's full size (the 256^3 torus, r_out = 1000 M,
a = 0.9375, gamma = 4/3, beta_0 = 100, as bench.py runs it), in the launch
configuration bench.py times (the step's own flux kernels: 16-face X1 / X2
columns, X3 row warps with a ragged last segment), on sampled outputs the
oracle computes one at a time:
  * Riemann fluxes of 6000 sampled faces against the oracle's single-face
    flux from the same four zone states (the oracle's (r, theta) metric
    records of a 256 x 256 grid: the metric does not depend on phi); with
    PPM faces (the bench's PPM step) from the same six zone states;
  * the inversion at 20000 sampled zones: the oracle's con2prim of the GPU's
    conserved variables, started from the GPU's primitives, returns them;
  * a property that holds at any size: the corner divergence of B (Eq. 24)
    stays at FP64 round-off of the flux-CT update, in both paths.
FP64: the 1e-10 parity bound.  Mixed: the faces are FP32, so the bound is
FP32 rounding through the face physics (1e-5 of each component's scale);
the mixed energy flux is compared rest-mass subtracted, as the mixed path
carries it."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import gpu_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 256
A, GAM, R_OUT = 0.9375, 4.0 / 3.0, 1000.0
NOT_B = [0, 1, 2, 3, 4, 8]


def _bench_torus(G, precision, steps, recon=0):
    gp = G.default_grid(N, N, N, a=A, r_out=R_OUT, precision=precision, recon=recon)
    ctx = G.init_grid(gp, G.default_phys(gam=GAM))
    G.set_metric(ctx, A, G.KERR_MKS)
    G.init_torus(ctx, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=3)
    G.step(ctx, steps)
    G.sync(ctx)
    return ctx


def _oracle_records(recon=0):
    return O.Grid(O.default_params(n1=N, n2=N, n3=1, a=A, r_out=R_OUT, gam=GAM, recon=recon))


def _sample_faces(rng, d, n, w=2):
    """face indices (i, j, k) of direction d whose stencil of 2 w zones
    (w = 2: PLM, 3: PPM) lies in the active zones (X3 wraps periodically),
    with the ends of the ranges always included"""
    lo = [0, 0, 0]
    hi = [N - 1, N - 1, N - 1]
    if d < 2:
        lo[d], hi[d] = w, N - w
    else:
        hi[2] = N  # faces 0 .. n3, stencils wrap in phi
    idx = np.stack([rng.integers(lo[e], hi[e] + 1, n) for e in range(3)], axis=1)
    ends = np.array([[lo[0], lo[1], lo[2]], [hi[0], hi[1], hi[2]]])
    return np.concatenate([ends, idx])


def _loc(faces, d, o):
    """metric record (i * n2 + j) of the zone at offset o along d from each face"""
    z = faces.copy()
    z[:, d] += o
    if d == 2:
        z[:, 2] %= N
    return (z[:, 0] * N + z[:, 1]).astype(np.int32)


@pytest.mark.parametrize("precision,recon", [(0, O.PLM), (1, O.PLM), (0, O.PPM), (1, O.PPM)])
def test_fullsize_face_fluxes(precision, recon):
    G = gpu_mod()
    w = 3 if recon == O.PPM else 2
    ctx = _bench_torus(G, precision, 3, recon)
    Pd = torch.empty((8, N, N, N), dtype=torch.float64, device="cuda")
    Ud = torch.empty((9, N, N, N), dtype=torch.float64, device="cuda")
    G.get_state(ctx, Pd, Ud)
    del Ud
    Fd = torch.zeros((3, 9, N + 1, N + 1, N + 1), dtype=torch.float64, device="cuda")
    G.fluxes(ctx, Fd)
    og = _oracle_records(recon)
    rng = np.random.default_rng(20260)
    for d in range(3):
        faces = _sample_faces(rng, d, 2000, w)
        fi = torch.as_tensor(faces, device="cuda")
        Fg = Fd[d][:, fi[:, 0], fi[:, 1], fi[:, 2]].cpu().numpy().T  # (n, 9)
        # the zone states of every stencil, gathered on the device
        sten = []
        for o in range(-w, w):
            z = faces.copy()
            z[:, d] += o
            if d == 2:
                z[:, 2] %= N
            zt = torch.as_tensor(z, device="cuda")
            sten.append(Pd[:, zt[:, 0], zt[:, 1], zt[:, 2]].cpu().numpy().T)  # (n, 8)
        sten = np.stack(sten, axis=1)  # (n, 2 w, 8)
        Fo, cw = [], []
        for m, f in enumerate(faces):
            F1, c1 = og.face_flux_at(d, f[0], f[1], sten[m])
            Fo.append(F1)
            cw.append(c1)
        Fo, cw = np.array(Fo), np.array(cw)
        if precision == 1:
            Fo[:, 1] += Fo[:, 0]  # rest-mass-subtracted energy flux
            # the LLF flux 1/2 (F_l + F_r - c_w (U_r - U_l)) rounds its terms: the
            # FP32 error of a face is eps_32 x (|F| + c_w |U|) times the depth of
            # the dependent arithmetic; U of the two zones next to the face (the
            # oracle's conserved variables at their centres) sets the scale
            Ul = og.prim2cons(np.ascontiguousarray(sten[:, w - 1].T), _loc(faces, d, -1))
            Ur = og.prim2cons(np.ascontiguousarray(sten[:, w].T), _loc(faces, d, 0))
            Ul[1] += Ul[0]
            Ur[1] += Ur[0]
            # (max-norm over the samples: where a component cancels to ~0, e.g.
            # the angular momentum flux of the static atmosphere, the rounding
            # of the cancelling terms is what remains on both sides)
            scale = np.abs(Fo) + cw[:, None] * np.maximum(np.abs(Ul), np.abs(Ur)).T
            errs = [np.abs(Fg[:, c] - Fo[:, c]).max() / scale[:, c].max() for c in NOT_B]
            print("direction", d + 1, "max-norm flux errors / (|F| + c_w |U|)", np.array(errs))
            assert max(errs) < 1e-5, (d, errs)
        else:
            errs = [np.abs(Fg[:, c] - Fo[:, c]).max() / np.abs(Fo[:, c]).max() for c in NOT_B]
            print("direction", d + 1, "max-norm relative flux errors", np.array(errs))
            assert max(errs) < 1e-10, (d, errs)
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_fullsize_inversion_and_div_b(precision):
    G = gpu_mod()
    ctx = _bench_torus(G, precision, 5)
    d = G.diagnostics(ctx)
    Pd = torch.empty((8, N, N, N), dtype=torch.float64, device="cuda")
    Ud = torch.empty((9, N, N, N), dtype=torch.float64, device="cuda")
    G.get_state(ctx, Pd, Ud)
    og = _oracle_records()
    rng = np.random.default_rng(7)
    n = 20000
    z = np.stack([rng.integers(0, N, n) for _ in range(3)], axis=1)
    # the polar interpolation of ut^2 in the two zones next to each pole acts
    # on P only (not U), so those zones are not a root of their own U
    z = z[(z[:, 1] >= 2) & (z[:, 1] < N - 2)]
    n = len(z)
    zt = torch.as_tensor(z, device="cuda")
    P = Pd[:, zt[:, 0], zt[:, 1], zt[:, 2]].cpu().numpy()
    U = Ud[:, zt[:, 0], zt[:, 1], zt[:, 2]].cpu().numpy()
    loc = (z[:, 0] * N + z[:, 1]).astype(np.int32)
    Pq, flags = og.con2prim(np.ascontiguousarray(U), loc, np.ascontiguousarray(P))[:2]
    assert np.all((flags & 8) == 0)  # the oracle inverts every sampled zone
    if precision == 0:
        # the GPU state is a root of its own U to the Newton tolerance
        sel, tol = np.ones(n, dtype=bool), 1e-9
    else:
        # torus body (no floors, whose FP32-assembled U carries the thermal
        # energy only to FP32 accuracy of the binding energy): the stored
        # primitives are the FP64 root of U rounded to FP32
        sel, tol = P[0] > 1e-4, 1e-6
    assert sel.sum() > 100
    # rho pointwise; u relative to rho + u (u = p/(gam-1) comes from
    # W (1 - v^2) - D sqrt(1 - v^2) = rho (h - 1), so a root's u is known to
    # eps x rho h, not eps x u, in cold gas); velocities max-norm
    errs = []
    for f in range(5):
        if f == 0:
            scale = np.abs(Pq[0, sel])
        elif f == 1:
            scale = np.abs(Pq[0, sel]) + np.abs(Pq[1, sel])
        else:
            scale = np.abs(Pq[f, sel]).max()
        errs.append((np.abs(P[f, sel] - Pq[f, sel]) / scale).max())
    print("round-trip errors rho, u, ut1..3:", np.array(errs))
    assert max(errs) < tol, errs
    # div B of Eq. 24 (corner sums of U_B x 1/dX) at FP64 round-off in both
    # paths: the mixed path's EMFs are FP32, but every face's CT flux is one
    # consistent value and the increments of U_B are formed in FP64
    ub = float(Ud[5:8].abs().max())
    idx = max(1.0 / og.dx[0], 1.0 / og.dx[1], N / (2 * np.pi))
    bound = 1e-12 * ub * idx
    print("div B max", d["divb_max"], "bound", bound)
    assert d["divb_max"] < bound
    ctx.close()
