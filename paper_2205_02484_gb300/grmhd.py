"""Thin ctypes binding of libgrmhd.so (include/grmhd.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be numpy arrays (host memory, on_device=0) or torch
CUDA tensors (device memory, on_device=1); shapes follow the header's
field-major active-zone layout.  Errors raise GrmhdError with the library's
message.  If the shared library is missing the import fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

KERR_MKS, MINK_CART = 0, 1
BC_INFLOW, BC_POLAR, BC_PERIODIC, BC_OUTFLOW, BC_EXTERNAL = 0, 1, 2, 3, 4
LLF, HLL = 0, 1
PLM, PPM = 0, 1
FP64, MIXED = 0, 1
C2P_NR, C2P_BRENT_W, C2P_ENTROPY, C2P_ENTROPY_BETA = 0, 1, 2, 3
C2P_FAIL, C2P_FAIL_D, C2P_FAIL_ENT, C2P_LEARNED = 8, 16, 32, 64
NP, NU = 8, 9
NG = 3  # ghost layers per side of the library's grids

EINVAL, ECUDA, ENOMEM, ENONFINITE, EFIXUP, EITER, ESTATE = -1, -2, -3, -4, -5, -6, -7
ERRORS = {-1: "EINVAL", -2: "ECUDA", -3: "ENOMEM", -4: "ENONFINITE", -5: "EFIXUP", -6: "EITER",
          -7: "ESTATE"}


class GrmhdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"grmhd {ERRORS.get(code, code)}: {msg}")
        self.code = code


class GridParams(C.Structure):
    _fields_ = [
        ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("metric", C.c_int),
        ("r_in", C.c_double), ("r_out", C.c_double), ("hslope", C.c_double), ("r_br", C.c_double),
        ("n_x", C.c_double), ("R0", C.c_double),
        ("x1min", C.c_double), ("x1max", C.c_double), ("x2min", C.c_double), ("x2max", C.c_double),
        ("x3min", C.c_double), ("x3max", C.c_double),
        ("bc1", C.c_int), ("bc2", C.c_int), ("bc3", C.c_int), ("riemann", C.c_int),
        ("precision", C.c_int), ("device", C.c_int), ("stream", C.c_void_p),
        ("j0", C.c_int), ("n2_total", C.c_int), ("recon", C.c_int),
        ("cyl_r", C.c_double), ("cyl_dx2", C.c_double),
    ]


class PhysParams(C.Structure):
    _fields_ = [("gam", C.c_double), ("cfl", C.c_double), ("nr_tol", C.c_double),
                ("sigma_max", C.c_double), ("bu_max", C.c_double), ("gamma_max", C.c_double),
                ("beta_entropy", C.c_double), ("nr_maxit", C.c_int), ("brent_maxit", C.c_int),
                ("fix_maxsweep", C.c_int)]


class TorusParams(C.Structure):
    _fields_ = [("r_in", C.c_double), ("r_max", C.c_double), ("beta0", C.c_double),
                ("pert_amp", C.c_double), ("kappa", C.c_double), ("seed", C.c_ulonglong)]


class Diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("t", "dt", "mdot", "phib", "PhiB", "edot", "ldot", "divb_max", "disk_mass", "disk_eb", "eta")] + \
               [(n, C.c_longlong) for n in
                ("nr_iters", "n_nr", "n_brent", "n_entropy", "n_entropy_beta", "n_fail", "n_floor",
                 "n_ceil", "n_gcap", "n_fixed", "fix_sweeps", "n_steps", "n_learned")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class EnsTiling(C.Structure):
    _fields_ = [("items_flux", C.c_int), ("items_update", C.c_int), ("blocks_per_sm_flux", C.c_int),
                ("blocks_per_sm_update", C.c_int), ("solo_log2", C.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


# every symbol include/grmhd.h declares, with its ctypes signature
_V = C.c_void_p
MLP_NPARAM = 4609
MLP_NNORM = 12


class MlpTrainParams(C.Structure):
    _fields_ = [("n_samples", C.c_long), ("n_val", C.c_long), ("seed", C.c_ulonglong),
                ("init_seed", C.c_ulonglong), ("epochs", C.c_int), ("batch", C.c_int),
                ("lr", C.c_double), ("lr_min", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double), ("weight_decay", C.c_double)]


class MlpTrainReport(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("val_rmse", C.c_double),
                ("val_maxerr", C.c_double), ("train_ms", C.c_double), ("samples_per_s", C.c_double),
                ("steps", C.c_long)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


SIGNATURES = {
    "grmhd_init_grid": (C.c_int, [C.POINTER(GridParams), C.POINTER(PhysParams), C.POINTER(_V)]),
    "grmhd_set_metric": (C.c_int, [_V, C.c_double, C.c_int]),
    "grmhd_init_torus": (C.c_int, [_V, C.POINTER(TorusParams)]),
    "grmhd_set_state": (C.c_int, [_V, _V, _V, C.c_double, C.c_double, C.c_int]),
    "grmhd_get_state": (C.c_int, [_V, _V, _V, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int]),
    "grmhd_set_state_u": (C.c_int, [_V, _V, C.c_double, C.c_double, C.c_int]),
    "grmhd_step": (C.c_int, [_V, C.c_int]),
    "grmhd_con2prim": (C.c_int, [_V, _V, _V, _V, _V, _V, C.c_long, C.c_int, C.c_int]),
    "grmhd_prim2cons": (C.c_int, [_V, _V, _V, _V, C.c_long, C.c_int]),
    "grmhd_fluxes": (C.c_int, [_V, _V, C.POINTER(C.c_double), C.c_int]),
    "grmhd_sync": (C.c_int, [_V]),
    "grmhd_diag_partials": (C.c_int, [_V, C.c_double, _V]),
    "grmhd_diag_combine": (C.c_int, [_V, _V, C.c_int, C.POINTER(Diag), C.POINTER(C.c_double)]),
    "grmhd_diagnostics": (C.c_int, [_V, C.POINTER(Diag)]),
    "grmhd_destroy": (None, [_V]),
    "grmhd_last_error": (C.c_char_p, [_V]),
    "grmhd_version": (C.c_char_p, []),
    "grmhd_step_profiled": (C.c_int, [_V, C.c_int, C.POINTER(C.c_double)]),
    "grmhd_peak_probe": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "grmhd_diagnostics_noalloc": (C.c_int, [_V, _V]),
    "grmhd_ensemble_create": (C.c_int, [C.POINTER(_V), C.c_int, C.POINTER(_V)]),
    "grmhd_ensemble_step": (C.c_int, [_V, C.c_int]),
    "grmhd_ensemble_set_tiling": (C.c_int, [_V, C.POINTER(EnsTiling)]),
    "grmhd_ensemble_get_tiling": (C.c_int, [_V, C.POINTER(EnsTiling)]),
    "grmhd_ensemble_autotune": (C.c_int, [_V, C.c_int, C.POINTER(EnsTiling), C.POINTER(C.c_double)]),
    "grmhd_ensemble_sync": (C.c_int, [_V]),
    "grmhd_ensemble_destroy": (None, [_V]),
    "grmhd_ensemble_last_error": (C.c_char_p, [_V]),
    "grmhd_mlp_load": (C.c_int, [_V, _V, _V]),
    "grmhd_mlp_get": (C.c_int, [_V, _V, _V]),
    "grmhd_mlp_samples": (C.c_int, [_V, C.c_ulonglong, C.c_long, C.c_long, _V, _V, _V, _V, _V, C.c_int]),
    "grmhd_mlp_forward": (C.c_int, [_V, _V, C.c_long, _V, C.c_int]),
    "grmhd_mlp_loss_grad": (C.c_int, [_V, _V, _V, _V, _V, C.c_long, _V, C.POINTER(C.c_double), C.c_int]),
    "grmhd_mlp_train_steps": (C.c_int, [_V, _V, _V, _V, _V, C.c_long, C.c_long, C.c_long, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.POINTER(C.c_double), C.c_int]),
    "grmhd_mlp_train": (C.c_int, [_V, C.POINTER(MlpTrainParams), C.POINTER(MlpTrainReport)]),
    "grmhd_set_learned_guess": (C.c_int, [_V, C.c_int]),
    "grmhd_barycentric_radius": (C.c_int, [_V, C.c_double, C.POINTER(C.c_double)]),
    "grmhd_stage": (C.c_int, [_V, C.c_int]),
    "grmhd_step_dtd": (C.c_int, [_V, _V, C.c_int]),
    "grmhd_finish_step": (C.c_int, [_V, _V]),
    "grmhd_x3_plane_bytes": (C.c_int, [_V, C.POINTER(C.c_ulonglong)]),
    "grmhd_x3_pack": (C.c_int, [_V, C.c_int, C.c_int, _V]),
    "grmhd_x3_unpack": (C.c_int, [_V, C.c_int, C.c_int, _V]),
    "grmhd_stage_update": (C.c_int, [_V, C.c_int]),
    "grmhd_fail_count": (C.c_int, [_V, _V]),
    "grmhd_fix_sweep": (C.c_int, [_V, C.c_int, _V]),
    "grmhd_fix_end": (C.c_int, [_V, C.c_int, C.c_int]),
    "grmhd_theta_ring_fix": (C.c_int, [C.POINTER(_V), C.c_int, C.c_int, _V]),
    "grmhd_stage_bc": (C.c_int, [_V, C.c_int]),
    "grmhd_x2_row_bytes": (C.c_int, [_V, C.c_int, C.POINTER(C.c_ulonglong)]),
    "grmhd_x2_pack": (C.c_int, [_V, C.c_int, C.c_int, C.c_int, _V]),
    "grmhd_x2_unpack": (C.c_int, [_V, C.c_int, C.c_int, C.c_int, _V]),
}

PROF_SLOTS = 16
PROF_PARTS = ("flux_x1", "flux_x2", "flux_x3", "emf", "update_c2p", "fixup", "bc")

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgrmhd.so (raises if it is missing and building is not allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} not built: run __graft_entry__.build() or "
                              f"python -m paper_2205_02484_gb300.build")
        _build.build()
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, 0
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr(), 1 if a.is_cuda else 0


class Context:
    """Owning handle of one grmhd_ctx."""

    def __init__(self, handle, grid: GridParams, phys: PhysParams):
        self.h = handle
        self.grid = grid
        self.phys = phys
        self.L = load()

    @property
    def shape(self):
        return (self.grid.n1, self.grid.n2, self.grid.n3)

    @property
    def nact(self):
        return self.grid.n1 * self.grid.n2 * self.grid.n3

    def check(self, rc):
        if rc != 0:
            msg = self.L.grmhd_last_error(self.h)
            raise GrmhdError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if self.h:
            self.L.grmhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_phys(gam=13.0 / 9.0, **kw) -> PhysParams:
    d = dict(gam=gam, cfl=0.45, nr_tol=1e-10, sigma_max=50.0, bu_max=2500.0, gamma_max=50.0,
             beta_entropy=1e-2, nr_maxit=30, brent_maxit=100, fix_maxsweep=16)
    d.update(kw)
    return PhysParams(**d)


def default_grid(n1, n2, n3, a=0.9375, r_out=40.0, precision=FP64, **kw) -> GridParams:
    d = dict(n1=n1, n2=n2, n3=n3, metric=KERR_MKS, r_in=0.98 * (1.0 + (1.0 - a * a) ** 0.5),
             r_out=r_out, hslope=0.3, r_br=400.0, n_x=4.0, R0=0.0, x1min=0.0, x1max=1.0, x2min=0.0,
             x2max=1.0, x3min=0.0, x3max=1.0, bc1=BC_OUTFLOW, bc2=BC_OUTFLOW, bc3=BC_PERIODIC,
             riemann=LLF, precision=precision, device=0, stream=None)
    d.update(kw)
    return GridParams(**d)


# ------------------------------------------------------------ ABI functions

def init_grid(grid: GridParams, phys: PhysParams) -> Context:
    L = load()
    h = C.c_void_p()
    rc = L.grmhd_init_grid(C.byref(grid), C.byref(phys), C.byref(h))
    if rc != 0:
        raise GrmhdError(rc, L.grmhd_last_error(None).decode())
    return Context(h.value, grid, phys)


def set_metric(ctx: Context, a: float, kind: int = KERR_MKS):
    ctx.check(ctx.L.grmhd_set_metric(ctx.h, a, kind))


def init_torus(ctx: Context, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=1, kappa=1e-3):
    tp = TorusParams(r_in, r_max, beta0, pert_amp, kappa, seed)
    ctx.check(ctx.L.grmhd_init_torus(ctx.h, C.byref(tp)))


def set_state(ctx: Context, P, U, t: float, dt: float):
    pp, dev = _ptr(P)
    up, dev2 = _ptr(U)
    if dev != dev2:
        raise ValueError("P and U must both be host or both be device")
    ctx.check(ctx.L.grmhd_set_state(ctx.h, pp, up, t, dt, dev))


def set_state_u(ctx: Context, U, t: float, dt: float):
    """The state from U (9, n1, n2, n3) alone; the primitives are re-derived on
    the device (numpy array = host, CUDA tensor = device)."""
    up, dev = _ptr(U)
    ctx.check(ctx.L.grmhd_set_state_u(ctx.h, up, t, dt, dev))


def get_state_u(ctx: Context, U=None):
    """Fills U (9, n1, n2, n3) alone (numpy or CUDA tensor; a new numpy array if
    None) and returns (U, t, dt)."""
    if U is None:
        U = np.zeros((NU,) + ctx.shape)
    up, dev = _ptr(U)
    t, dt = C.c_double(), C.c_double()
    ctx.check(ctx.L.grmhd_get_state(ctx.h, None, up, C.byref(t), C.byref(dt), dev))
    return U, t.value, dt.value


def get_state(ctx: Context, P=None, U=None):
    """Fills P (8, n1, n2, n3) and U (9, ...) (numpy or CUDA tensors; new numpy
    arrays if None) and returns (P, U, t, dt)."""
    if P is None:
        P = np.zeros((NP,) + ctx.shape)
    if U is None:
        U = np.zeros((NU,) + ctx.shape)
    pp, dev = _ptr(P)
    up, dev2 = _ptr(U)
    if dev != dev2:
        raise ValueError("P and U must both be host or both be device")
    t, dt = C.c_double(), C.c_double()
    ctx.check(ctx.L.grmhd_get_state(ctx.h, pp, up, C.byref(t), C.byref(dt), dev))
    return P, U, t.value, dt.value


def step(ctx: Context, nsteps: int = 1):
    ctx.check(ctx.L.grmhd_step(ctx.h, nsteps))


# ------------------------------------------------- phi slabs (stage level)

def _dev_ptr(t):
    p, dev = _ptr(t)
    if not dev:
        raise ValueError("a device tensor is required")
    return p


def stage(ctx: Context, st: int):
    """One RK2 stage: 0 predictor, 1 corrector (Eqs. 25-26)."""
    ctx.check(ctx.L.grmhd_stage(ctx.h, st))


def step_dtd(ctx: Context, dtd, accumulate: bool = False):
    """The last predictor's per-direction CFL minima into dtd (3 doubles on
    the device), stored or folded in by a minimum."""
    ctx.check(ctx.L.grmhd_step_dtd(ctx.h, _dev_ptr(dtd), int(bool(accumulate))))


def finish_step(ctx: Context, dtd):
    """Advance t by dt and set the next dt from Eq. 27 over dtd (3 doubles on the device)."""
    ctx.check(ctx.L.grmhd_finish_step(ctx.h, _dev_ptr(dtd)))


def x3_plane_bytes(ctx: Context) -> int:
    n = C.c_ulonglong(0)
    ctx.check(ctx.L.grmhd_x3_plane_bytes(ctx.h, C.byref(n)))
    return n.value


def _buf_ptr(buf, nbytes):
    if buf.numel() * buf.element_size() < nbytes:
        raise ValueError(f"buffer of {buf.numel() * buf.element_size()} bytes < {nbytes}")
    return _dev_ptr(buf)


def x3_pack(ctx: Context, which: int, side: int, buf):
    ctx.check(ctx.L.grmhd_x3_pack(ctx.h, which, side, _buf_ptr(buf, x3_plane_bytes(ctx))))


def x3_unpack(ctx: Context, which: int, side: int, buf):
    ctx.check(ctx.L.grmhd_x3_unpack(ctx.h, which, side, _buf_ptr(buf, x3_plane_bytes(ctx))))


# ----------------------------------------------- theta slabs (stage parts)

def _acc_ptr(acc):
    import torch
    if acc.dtype != torch.int64 or acc.numel() < 1:
        raise ValueError("the count accumulator is one int64 on the device")
    return _dev_ptr(acc)


def stage_update(ctx: Context, st: int):
    """Fluxes, flux-CT, update and inversion of stage st (up to its fixups)."""
    ctx.check(ctx.L.grmhd_stage_update(ctx.h, st))


def fail_count(ctx: Context, acc):
    """Add the number of failed inversions of the last stage_update to acc (int64 on the device)."""
    ctx.check(ctx.L.grmhd_fail_count(ctx.h, _acc_ptr(acc)))


def fix_sweep(ctx: Context, st: int, acc):
    """One fixup sweep (Eq. 33) of stage st; adds the zones still failed to acc."""
    ctx.check(ctx.L.grmhd_fix_sweep(ctx.h, st, _acc_ptr(acc)))


def fix_end(ctx: Context, st: int, nsweeps: int):
    ctx.check(ctx.L.grmhd_fix_end(ctx.h, st, nsweeps))


def theta_ring_fix(ctxs, st: int, nsweeps=None):
    """The fixup loop of stage st over the theta slabs `ctxs` of one grid on
    one device (theta order), run on the device; nsweeps: an int32 device
    tensor that receives the sweep count, or None."""
    import torch
    if nsweeps is not None and (nsweeps.dtype != torch.int32 or nsweeps.numel() < 1):
        raise ValueError("nsweeps must be an int32 device tensor")
    hs = (_V * len(ctxs))(*[c.h for c in ctxs])
    ctxs[0].check(ctxs[0].L.grmhd_theta_ring_fix(hs, len(ctxs), st, None if nsweeps is None else _dev_ptr(nsweeps)))


def stage_bc(ctx: Context, st: int):
    ctx.check(ctx.L.grmhd_stage_bc(ctx.h, st))


def x2_row_bytes(ctx: Context, kind: int) -> int:
    """Bytes of one side's rows: kind 0 the NG ghost rows, kind 1 a fixup sweep's edge row."""
    n = C.c_ulonglong(0)
    ctx.check(ctx.L.grmhd_x2_row_bytes(ctx.h, kind, C.byref(n)))
    return n.value


def x2_pack(ctx: Context, kind: int, which: int, side: int, buf):
    ctx.check(ctx.L.grmhd_x2_pack(ctx.h, kind, which, side, _buf_ptr(buf, x2_row_bytes(ctx, kind))))


def x2_unpack(ctx: Context, kind: int, which: int, side: int, buf):
    ctx.check(ctx.L.grmhd_x2_unpack(ctx.h, kind, which, side, _buf_ptr(buf, x2_row_bytes(ctx, kind))))


DIAG_NPART = 26


def diag_partials(ctx: Context, r_bar_max: float, out):
    """This context's partial diagnostics (DIAG_NPART doubles) into the device
    tensor out, asynchronously on the context stream."""
    ctx.check(ctx.L.grmhd_diag_partials(ctx.h, float(r_bar_max), _dev_ptr(out)))


def diag_combine(ctx: Context, parts):
    """Whole-grid diagnostics from partial vectors parts (nparts x DIAG_NPART,
    a contiguous device tensor), added in their order on the device: (dict,
    (barycentric radius, mass sum, numerator))."""
    if parts.dim() != 2 or parts.shape[1] != DIAG_NPART:
        raise ValueError("parts must be (nparts, DIAG_NPART)")
    d = Diag()
    b = (C.c_double * 3)()
    ctx.check(ctx.L.grmhd_diag_combine(ctx.h, _dev_ptr(parts), int(parts.shape[0]), C.byref(d), b))
    return d.as_dict(), (b[0], b[1], b[2])


def sync(ctx: Context):
    ctx.check(ctx.L.grmhd_sync(ctx.h))


def diagnostics(ctx: Context) -> dict:
    d = Diag()
    ctx.check(ctx.L.grmhd_diagnostics(ctx.h, C.byref(d)))
    return d.as_dict()


def barycentric_radius(ctx: Context, r_bar_max: float = 80.0):
    """(<r>, mass sum, numerator) of Eq. 43 over r_H <= r <= r_bar_max."""
    out = (C.c_double * 3)()
    ctx.check(ctx.L.grmhd_barycentric_radius(ctx.h, float(r_bar_max), out))
    return tuple(out)


def prim2cons(ctx: Context, P, loc, U=None):
    n = loc.shape[0]
    if U is None:
        U = np.zeros((NU, n))
    pp, dev = _ptr(P)
    lp, _ = _ptr(loc)
    up, _ = _ptr(U)
    ctx.check(ctx.L.grmhd_prim2cons(ctx.h, pp, lp, up, n, dev))
    return U


def con2prim(ctx: Context, U, loc, P_inout, flags=None, iters=None, use_learned_guess=False):
    n = loc.shape[0]
    if flags is None:
        flags = np.zeros(n, dtype=np.int32)
    if iters is None:
        iters = np.zeros(n, dtype=np.int32)
    up, dev = _ptr(U)
    lp, _ = _ptr(loc)
    pp, _ = _ptr(P_inout)
    fp, _ = _ptr(flags)
    ip, _ = _ptr(iters)
    ctx.check(ctx.L.grmhd_con2prim(ctx.h, up, lp, pp, fp, ip, n, int(use_learned_guess), dev))
    return P_inout, flags, iters


def fluxes(ctx: Context, out=None):
    n1, n2, n3 = ctx.shape
    if out is None:
        out = np.zeros((3, NU, n1 + 1, n2 + 1, n3 + 1))
    op, dev = _ptr(out)
    dt = C.c_double()
    ctx.check(ctx.L.grmhd_fluxes(ctx.h, op, C.byref(dt), dev))
    return out, dt.value


def step_profiled(ctx: Context, nsteps: int = 1) -> dict:
    """Per-kernel-group milliseconds summed over nsteps (CUDA events on the
    context stream); keys '<part>_pred', '<part>_corr', 'finalize', 'step'."""
    buf = (C.c_double * PROF_SLOTS)()
    ctx.check(ctx.L.grmhd_step_profiled(ctx.h, nsteps, buf))
    out = {}
    for st, tag in ((0, "pred"), (1, "corr")):
        for p, name in enumerate(PROF_PARTS):
            out[f"{name}_{tag}"] = buf[st * 7 + p]
    out["finalize"] = buf[14]
    out["step"] = buf[15]
    return out


def diagnostics_noalloc(ctx: Context, out_dev):
    """Horizon diagnostics into a caller-owned CUDA tensor of 8 doubles
    without any device allocation (asynchronous on the context stream)."""
    ptr, dev = _ptr(out_dev)
    if not dev or out_dev.numel() < 8:
        raise ValueError("out_dev must be a CUDA tensor of at least 8 doubles")
    ctx.check(ctx.L.grmhd_diagnostics_noalloc(ctx.h, ptr))
    return out_dev


# ------------------------------------------------------------------ ensemble

class Ensemble:
    """Owning handle of a grmhd_ens; keeps its member contexts alive."""

    def __init__(self, handle, members):
        self.h = handle
        self.members = list(members)
        self.L = load()

    def check(self, rc):
        if rc != 0:
            msg = self.L.grmhd_ensemble_last_error(self.h) if self.h else b""
            raise GrmhdError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if self.h:
            self.L.grmhd_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ensemble_create(members) -> Ensemble:
    L = load()
    arr = (C.c_void_p * len(members))(*[m.h for m in members])
    h = C.c_void_p()
    rc = L.grmhd_ensemble_create(arr, len(members), C.byref(h))
    if rc != 0:
        raise GrmhdError(rc, "ensemble_create failed (members must share device and precision and have a state)")
    return Ensemble(h.value, members)


def ensemble_step(ens: Ensemble, nsteps: int = 1):
    ens.check(ens.L.grmhd_ensemble_step(ens.h, nsteps))


def ensemble_sync(ens: Ensemble):
    ens.check(ens.L.grmhd_ensemble_sync(ens.h))


def ensemble_set_tiling(ens: Ensemble, items_flux, items_update, blocks_per_sm_flux, blocks_per_sm_update,
                        solo_log2=0):
    """solo_log2 > 0: members of at least 2**solo_log2 active zones step with
    their own kernels inside the ensemble graph."""
    t = EnsTiling(items_flux, items_update, blocks_per_sm_flux, blocks_per_sm_update, solo_log2)
    ens.check(ens.L.grmhd_ensemble_set_tiling(ens.h, C.byref(t)))


def ensemble_get_tiling(ens: Ensemble) -> dict:
    t = EnsTiling()
    ens.check(ens.L.grmhd_ensemble_get_tiling(ens.h, C.byref(t)))
    return t.as_dict()


def ensemble_autotune(ens: Ensemble, trial_steps: int = 2):
    t = EnsTiling()
    ms = C.c_double()
    ens.check(ens.L.grmhd_ensemble_autotune(ens.h, trial_steps, C.byref(t), C.byref(ms)))
    return t.as_dict(), ms.value


def peak_probe(device: int = 0, fp64: bool = True) -> float:
    L = load()
    v = C.c_double()
    rc = L.grmhd_peak_probe(device, int(fp64), C.byref(v))
    if rc != 0:
        raise GrmhdError(rc, L.grmhd_last_error(None).decode())
    return v.value


def version() -> str:
    return load().grmhd_version().decode()


# ------------------------------------------------------------ learned start

def _f32_host(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def mlp_load(ctx: Context, theta, norm):
    th = _f32_host(theta, MLP_NPARAM)
    nm = _f32_host(norm, MLP_NNORM)
    ctx.check(ctx.L.grmhd_mlp_load(ctx.h, th.ctypes.data, nm.ctypes.data))


def mlp_get(ctx: Context):
    th = np.zeros(MLP_NPARAM, dtype=np.float32)
    nm = np.zeros(MLP_NNORM, dtype=np.float32)
    ctx.check(ctx.L.grmhd_mlp_get(ctx.h, th.ctypes.data, nm.ctypes.data))
    return th, nm


def mlp_samples(ctx: Context, seed: int, first: int, n: int, device=False):
    """Samples first..first+n-1 of the seeded training distribution:
    P (8, n), loc (n), U (9, n), feat (5, n) FP32, label (n) FP32."""
    if device:
        import torch
        dev = torch.device("cuda", ctx.grid.device)
        P = torch.zeros((NP, n), dtype=torch.float64, device=dev)
        loc = torch.zeros(n, dtype=torch.int32, device=dev)
        U = torch.zeros((NU, n), dtype=torch.float64, device=dev)
        feat = torch.zeros((5, n), dtype=torch.float32, device=dev)
        lab = torch.zeros(n, dtype=torch.float32, device=dev)
    else:
        P, loc, U = np.zeros((NP, n)), np.zeros(n, dtype=np.int32), np.zeros((NU, n))
        feat, lab = np.zeros((5, n), dtype=np.float32), np.zeros(n, dtype=np.float32)
    ptrs = [_ptr(a)[0] for a in (P, loc, U, feat, lab)]
    ctx.check(ctx.L.grmhd_mlp_samples(ctx.h, seed, first, n, *ptrs, int(device)))
    return P, loc, U, feat, lab


def mlp_forward(ctx: Context, feat, y=None):
    n = feat.shape[-1]
    if y is None:
        y = np.zeros(n, dtype=np.float32)
    fp, dev = _ptr(feat)
    yp, _ = _ptr(y)
    ctx.check(ctx.L.grmhd_mlp_forward(ctx.h, fp, n, yp, dev))
    return y


def mlp_loss_grad(ctx: Context, theta, norm, feat, label):
    th = _f32_host(theta, MLP_NPARAM)
    nm = _f32_host(norm, MLP_NNORM)
    n = feat.shape[-1]
    fp, dev = _ptr(feat)
    lp, _ = _ptr(label)
    if dev:
        import torch
        grad = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=feat.device)
    else:
        grad = np.zeros(MLP_NPARAM, dtype=np.float32)
    gp, _ = _ptr(grad)
    loss = C.c_double()
    ctx.check(ctx.L.grmhd_mlp_loss_grad(ctx.h, th.ctypes.data, nm.ctypes.data, fp, lp, n, gp, C.byref(loss), dev))
    return loss.value, grad


def mlp_train_steps(ctx: Context, theta, norm, feat, label, batch, nsteps, lr, beta1=0.9, beta2=0.999,
                    eps=1e-8, weight_decay=0.0):
    th = _f32_host(theta, MLP_NPARAM).copy()
    nm = _f32_host(norm, MLP_NNORM)
    n = feat.shape[-1]
    fp, dev = _ptr(feat)
    lp, _ = _ptr(label)
    loss = C.c_double()
    ctx.check(ctx.L.grmhd_mlp_train_steps(ctx.h, th.ctypes.data, nm.ctypes.data, fp, lp, n, batch, nsteps, lr,
                                          beta1, beta2, eps, weight_decay, C.byref(loss), dev))
    return th, loss.value


def mlp_train(ctx: Context, n_samples=10_000_000, n_val=100_000, seed=7, init_seed=1, epochs=4, batch=4096,
              lr=2e-3, lr_min=2e-5, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4) -> dict:
    tp = MlpTrainParams(n_samples, n_val, seed, init_seed, epochs, batch, lr, lr_min, beta1, beta2, eps,
                        weight_decay)
    rep = MlpTrainReport()
    ctx.check(ctx.L.grmhd_mlp_train(ctx.h, C.byref(tp), C.byref(rep)))
    return rep.as_dict()


def set_learned_guess(ctx: Context, on: bool = True):
    ctx.check(ctx.L.grmhd_set_learned_guess(ctx.h, int(on)))
