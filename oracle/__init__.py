"""Plain FP64 CPU oracle of the cuHARM GR-MHD step (arXiv 2205.02484).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference that the CUDA path is compared with.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the product package and never imports it.

The C sources (``*.c`` next to this file) follow the paper section by section;
this module only compiles them with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["geometry.c", "physics.c", "con2prim.c", "grid.c", "torus.c", "mlp.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_CNT_PATH = os.path.join(_HERE, "libopcount.so")
_lock = threading.Lock()
_lib = None

NP, NU = 8, 9
NG = 3  # ghost layers per side (ORC_NG)
PLM, PPM = 0, 1  # reconstruction: Eqs. 16-17, or the parabolic method of Section 2.2
KERR_MKS, MINK_CART = 0, 1
BC_INFLOW, BC_POLAR, BC_PERIODIC, BC_OUTFLOW, BC_EXTERNAL = 0, 1, 2, 3, 4
LLF, HLL = 0, 1
C2P_NR, C2P_BRENT_W, C2P_ENTROPY, C2P_ENTROPY_BETA = 0, 1, 2, 3
C2P_FAIL, C2P_FAIL_D, C2P_FAIL_ENT = 8, 16, 32


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        deps = srcs + [os.path.join(_HERE, "orc.h")]
        if all(os.path.getmtime(s) <= lib_m for s in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    build_counter(force=True)
    return _LIB_PATH


def build_counter(force: bool = False) -> str:
    """Compile libopcount.so: the oracle's physics.c and con2prim.c compiled
    again as C++ with an operation-counting scalar (opcount.cpp)."""
    deps = [os.path.join(_HERE, s) for s in ("opcount.cpp", "physics.c", "con2prim.c", "orc.h")]
    if not force and os.path.exists(_CNT_PATH):
        if all(os.path.getmtime(s) <= os.path.getmtime(_CNT_PATH) for s in deps):
            return _CNT_PATH
    tmp = _CNT_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, "opcount.cpp"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _CNT_PATH)
    return _CNT_PATH


_cnt = None


def count_con2prim(U, geom34, guess, gam, methods=15, nr_tol=1e-10, beta_entropy=1e-2, nr_maxit=30,
                   brent_maxit=100, wguess=0.0):
    """The oracle's inversion of one state (Section 2.3) with its floating
    point operations counted: (flag, P, iters, counts) where counts has
    add, mul, div, sqrt, special (pow/exp/log calls) and flops (add + mul +
    div + sqrt).  geom34: gcov (16), gcon (16), sqrt(-g), alpha; wguess > 0:
    Newton first starts from that W."""
    global _cnt
    with _lock:
        if _cnt is None:
            build_counter()
            L = C.CDLL(_CNT_PATH)
            f = L.orc_count_con2prim
            f.restype = C.c_int
            f.argtypes = [_D, _D, _D, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                          C.c_double, _D, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
            _cnt = L
    U = np.ascontiguousarray(U, dtype=np.float64)
    g = np.ascontiguousarray(geom34, dtype=np.float64)
    q = np.ascontiguousarray(guess, dtype=np.float64)
    P = np.zeros(NP)
    it = C.c_int(0)
    out = (C.c_longlong * 6)()
    fl = _cnt.orc_count_con2prim(_p(U), _p(g), _p(q), gam, nr_tol, beta_entropy, nr_maxit, brent_maxit,
                                 methods, float(wguess), _p(P), C.byref(it), out)
    keys = ("add", "mul", "div", "sqrt", "special", "flops")
    return fl, P, it.value, dict(zip(keys, (int(v) for v in out)))


class Params(C.Structure):
    _fields_ = [
        ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("metric", C.c_int),
        ("a", C.c_double),
        ("r_in", C.c_double), ("r_out", C.c_double), ("hslope", C.c_double), ("r_br", C.c_double),
        ("n_x", C.c_double), ("R0", C.c_double),
        ("x1min", C.c_double), ("x1max", C.c_double), ("x2min", C.c_double), ("x2max", C.c_double),
        ("x3min", C.c_double), ("x3max", C.c_double),
        ("bc1", C.c_int), ("bc2", C.c_int), ("bc3", C.c_int), ("riemann", C.c_int),
        ("gam", C.c_double), ("cfl", C.c_double), ("nr_tol", C.c_double), ("sigma_max", C.c_double),
        ("bu_max", C.c_double), ("gamma_max", C.c_double), ("beta_entropy", C.c_double),
        ("nr_maxit", C.c_int), ("brent_maxit", C.c_int), ("fix_maxsweep", C.c_int),
        ("j0", C.c_int), ("n2_total", C.c_int), ("recon", C.c_int),
        ("cyl_r", C.c_double), ("cyl_dx2", C.c_double),
    ]


class TorusParams(C.Structure):
    _fields_ = [("r_in", C.c_double), ("r_max", C.c_double), ("beta0", C.c_double),
                ("pert_amp", C.c_double), ("kappa", C.c_double), ("seed", C.c_uint64)]


class Geom(C.Structure):
    _fields_ = [("gcov", C.c_double * 16), ("gcon", C.c_double * 16), ("gdet", C.c_double),
                ("alpha", C.c_double)]


class Diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("t", "dt", "mdot", "phib", "PhiB", "edot", "ldot", "divb_max", "disk_mass", "disk_eb", "eta")] + \
               [(n, C.c_longlong) for n in
                ("nr_iters", "n_nr", "n_brent", "n_entropy", "n_entropy_beta", "n_fail", "n_floor",
                 "n_ceil", "n_gcap", "n_fixed", "fix_sweeps", "n_steps")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_F = C.POINTER(C.c_float)


def _p(a: np.ndarray, t=_D):
    return a.ctypes.data_as(t)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            V = C.c_void_p
            sig = {
                "orc_create": (V, [C.POINTER(Params)]),
                "orc_destroy": (None, [V]),
                "orc_init_torus": (C.c_int, [V, C.POINTER(TorusParams)]),
                "orc_set_state": (None, [V, _D, _D, C.c_double, C.c_double]),
                "orc_get_state": (None, [V, _D, _D, _D, _D]),
                "orc_step": (C.c_int, [V]),
                "orc_initial_dt": (C.c_double, [V]),
                "orc_invert_all": (C.c_int, [V]),
                "orc_set_dt": (None, [V, C.c_double]),
                "orc_fluxes": (C.c_double, [V, _D]),
                "orc_diagnostics": (None, [V, C.POINTER(Diag)]),
                "orc_barycentric": (C.c_double, [V, C.c_double, _D]),
                "orc_face_flux_at": (C.c_double, [V, C.c_int, C.c_int, C.c_int, _D, _D]),
                "orc_p2c_batch": (None, [V, _D, _I, _D, C.c_long]),
                "orc_c2p_batch": (None, [V, _D, _I, _D, _D, _I, _I, C.c_long, C.c_int]),
                "orc_geom_table": (None, [V, C.c_int, _D]),
                "orc_conn_table": (None, [V, _D]),
                "orc_grid_info": (None, [V, _D]),
                "orc_get_flags": (None, [V, _I]),
                "orc_geom_at": (C.c_int, [V, C.c_double, C.c_double, C.POINTER(Geom)]),
                "orc_conn_at": (None, [V, C.c_double, C.c_double, _D]),
                "orc_r_of_x1": (C.c_double, [V, C.c_double]),
                "orc_th_of_x2": (C.c_double, [V, C.c_double]),
                "orc_theta_at": (C.c_double, [V, C.c_double, C.c_double, C.POINTER(C.c_double)]),
                "orc_ks_gcov": (None, [C.c_double, C.c_double, C.c_double, _D]),
                "orc_invert4": (C.c_int, [_D, _D, _D]),
                "orc_mc_slope": (C.c_double, [C.c_double, C.c_double, C.c_double]),
                "orc_state_of": (None, [_D, C.POINTER(Geom), _D]),
                "orc_prim_to_U": (None, [_D, C.POINTER(Geom), _D, C.c_double, _D]),
                "orc_prim_to_F": (None, [_D, C.POINTER(Geom), _D, C.c_double, C.c_int, _D]),
                "orc_wave_speeds": (None, [_D, C.POINTER(Geom), _D, C.c_double, C.c_int, _D, _D]),
                "orc_fm_lnh": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
                "orc_fm_ell": (C.c_double, [C.c_double, C.c_double]),
                "orc_fm_ucon_bl": (None, [C.c_double, C.c_double, C.c_double, C.c_double, _D]),
                "orc_uniform": (C.c_double, [C.c_uint64, C.c_uint64]),
                "orc_x1_of_r": (C.c_double, [V, C.c_double]),
                "orc_stage0": (C.c_double, [V, _I]),
                "orc_last_dtd": (None, [V, _D]),
                "orc_combine_dt": (C.c_double, [_D]),
                "orc_stage1": (None, [V, _I]),
                "orc_get_xplane": (None, [V, C.c_int, C.c_int, _D]),
                "orc_stage_update": (C.c_double, [V, C.c_int]),
                "orc_fail_count": (C.c_long, [V]),
                "orc_fix_sweep": (C.c_long, [V, C.c_int]),
                "orc_fix_end": (None, [V, C.c_int]),
                "orc_stage_bc": (None, [V, C.c_int]),
                "orc_get_yrow": (None, [V, C.c_int, C.c_int, _D]),
                "orc_set_yrow": (None, [V, C.c_int, C.c_int, _D]),
                "orc_get_fixrow": (None, [V, C.c_int, C.c_int, _D]),
                "orc_set_fixrow": (None, [V, C.c_int, C.c_int, _D]),
                "orc_set_xplane": (None, [V, C.c_int, C.c_int, _D]),
                "orc_mlp_nparam": (C.c_int, []),
                "orc_bf16_round": (C.c_float, [C.c_float]),
                "orc_mlp_features": (C.c_int, [_D, C.POINTER(Geom), _D]),
                "orc_mlp_samples": (None, [V, C.c_uint64, C.c_long, C.c_long, _D, _I, _D, _D, _D]),
                "orc_mlp_forward": (None, [_F, _F, _F, C.c_long, _D]),
                "orc_mlp_loss_grad": (C.c_double, [_F, _F, _F, _F, C.c_long, _D]),
                "orc_mlp_loss_grad_d": (C.c_double, [_D, _F, _F, _F, C.c_long, _D]),
                "orc_mlp_adamw": (None, [_D, _D, _D, _D, C.c_long, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double]),
                "orc_mlp_train_steps": (C.c_double, [_F, _F, _F, _F, C.c_long, C.c_long, C.c_long,
                                                     C.c_double, C.c_double, C.c_double, C.c_double,
                                                     C.c_double, _F, _F, _D]),
                "orc_c2p_batch_w": (None, [V, _D, _I, _D, _D, _D, _I, _I, C.c_long, C.c_int]),
                "orc_post_inversion_at": (None, [V, C.c_int, C.c_int, _D, _D, _I]),
                "orc_ppm_face": (None, [_D, _D]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def default_params(**kw) -> Params:
    """Physics defaults from the paper: cfl 0.45 (Eq. 27), Newton tolerance
    1e-10 (Section 2.3), b^2/rho < 50 and b^2/u < 2500, Gamma <= 50 and the
    beta < 1e-2 entropy switch (Section 2.4); MKS h = 0.3, n_X = 4, R0 = 0 and
    the hyper-exponential break at r = 400 M (Section 4.1)."""
    d = dict(n1=64, n2=64, n3=1, metric=KERR_MKS, a=0.9375, r_in=0.0, r_out=40.0, hslope=0.3,
             r_br=400.0, n_x=4.0, R0=0.0, x1min=0.0, x1max=1.0, x2min=0.0, x2max=1.0,
             x3min=0.0, x3max=1.0, bc1=BC_OUTFLOW, bc2=BC_OUTFLOW, bc3=BC_PERIODIC,
             riemann=LLF, gam=13.0 / 9.0, cfl=0.45, nr_tol=1e-10, sigma_max=50.0, bu_max=2500.0,
             gamma_max=50.0, beta_entropy=1e-2, nr_maxit=30, brent_maxit=100, fix_maxsweep=16, recon=PLM,
             cyl_r=0.0, cyl_dx2=0.0)
    d.update(kw)
    if d["r_in"] <= 0.0 and d["metric"] == KERR_MKS:
        d["r_in"] = 0.98 * (1.0 + (1.0 - d["a"] ** 2) ** 0.5)
    return Params(**d)


class Grid:
    """Owning wrapper around an oracle grid."""

    def __init__(self, params: Params):
        self.L = lib()
        self.p = params
        self.h = self.L.orc_create(C.byref(params))
        if not self.h:
            raise ValueError("oracle: bad grid parameters")
        info = np.zeros(10)
        self.L.orc_grid_info(self.h, _p(info))
        self.x1in, self.x2in, self.x3in = info[0:3]
        self.dx = info[3:6].copy()
        self.i_h = int(info[6])
        self.N = tuple(int(v) for v in info[7:10])
        self.ng = (self.N[0] - params.n1) // 2  # ghost layers per side
        assert self.ng == NG
        self.shape = (params.n1, params.n2, params.n3)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    @property
    def nact(self):
        return self.p.n1 * self.p.n2 * self.p.n3

    def init_torus(self, r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.04, seed=1, kappa=1e-3):
        tp = TorusParams(r_in, r_max, beta0, pert_amp, kappa, seed)
        rc = self.L.orc_init_torus(self.h, C.byref(tp))
        if rc != 0:
            raise RuntimeError(f"oracle init_torus failed: {rc}")

    def set_state(self, P, U, t, dt):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(NP, -1)
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(NU, -1)
        self.L.orc_set_state(self.h, _p(P), _p(U), float(t), float(dt))

    def get_state(self):
        P = np.zeros((NP,) + self.shape)
        U = np.zeros((NU,) + self.shape)
        t, dt = C.c_double(), C.c_double()
        self.L.orc_get_state(self.h, _p(P), _p(U), C.byref(t), C.byref(dt))
        return P, U, t.value, dt.value

    def step(self, n=1):
        st = 0
        for _ in range(n):
            st = self.L.orc_step(self.h) or st
        return st

    def set_dt(self, dt):
        self.L.orc_set_dt(self.h, float(dt))

    # ---- one slab of a phi-decomposed grid (bc3 = BC_EXTERNAL)
    def stage0(self):
        """Predictor stage; returns (dt candidate of this slab, status)."""
        st = C.c_int(0)
        dtn = self.L.orc_stage0(self.h, C.byref(st))
        return dtn, st.value

    def last_dtd(self):
        """Per-direction CFL minima of the last flux sweep."""
        out = np.zeros(3)
        self.L.orc_last_dtd(self.h, _p(out))
        return out

    def stage1(self):
        """Corrector stage (advances t); returns the status."""
        st = C.c_int(0)
        self.L.orc_stage1(self.h, C.byref(st))
        return st.value

    def xplane(self, which, k):
        """(8, N1, N2) primitives of P (which 0) or P-hat (which 1) at local X3 index k."""
        out = np.zeros((NP, self.N[0], self.N[1]))
        self.L.orc_get_xplane(self.h, which, k, _p(out))
        return out

    def set_xplane(self, which, k, plane):
        plane = np.ascontiguousarray(plane, dtype=np.float64)
        self.L.orc_set_xplane(self.h, which, k, _p(plane))

    # ---- one slab of a theta-decomposed grid (n2_total > 0)
    def stage_update(self, st):
        """Fluxes, flux-CT, update and inversion of stage st; returns this
        slab's CFL step (meaningful for st 0)."""
        return self.L.orc_stage_update(self.h, st)

    def fail_count(self):
        return int(self.L.orc_fail_count(self.h))

    def fix_sweep(self, st):
        """One fixup sweep over stage st's output; returns the zones still failed."""
        return int(self.L.orc_fix_sweep(self.h, st))

    def fix_end(self, nsweeps):
        self.L.orc_fix_end(self.h, nsweeps)

    def stage_bc(self, st):
        """Boundary fill of stage st's output (st 1 advances t)."""
        self.L.orc_stage_bc(self.h, st)

    def yrow(self, which, j):
        """(8, N1, N3) primitives of P (which 0) or P-hat (which 1) at local X2 index j."""
        out = np.zeros((NP, self.N[0], self.N[2]))
        self.L.orc_get_yrow(self.h, which, j, _p(out))
        return out

    def set_yrow(self, which, j, row):
        row = np.ascontiguousarray(row, dtype=np.float64)
        self.L.orc_set_yrow(self.h, which, j, _p(row))

    def fixrow(self, which, j):
        """(6, n1, n3): the five averaged primitives and the failure flag of row j."""
        out = np.zeros((6, self.p.n1, self.p.n3))
        self.L.orc_get_fixrow(self.h, which, j, _p(out))
        return out

    def set_fixrow(self, which, j, row):
        row = np.ascontiguousarray(row, dtype=np.float64)
        self.L.orc_set_fixrow(self.h, which, j, _p(row))

    def invert_all(self):
        return self.L.orc_invert_all(self.h)

    def initial_dt(self):
        return self.L.orc_initial_dt(self.h)

    def fluxes(self):
        m = (self.p.n1 + 1, self.p.n2 + 1, self.p.n3 + 1)
        out = np.zeros((3, NU) + m)
        dt = self.L.orc_fluxes(self.h, _p(out))
        return out, dt

    def diagnostics(self) -> dict:
        d = Diag()
        self.L.orc_diagnostics(self.h, C.byref(d))
        return d.as_dict()

    def barycentric(self, r_bar_max=80.0):
        """(<r>, mass sum, numerator) of Eq. 43 over r_H <= r <= r_bar_max."""
        out = np.zeros(3)
        self.L.orc_barycentric(self.h, float(r_bar_max), _p(out))
        return tuple(out)

    def face_flux_at(self, d, i, j, q4):
        """(F[9], c_w) of the Riemann flux of a face of direction d (0..2) at
        metric record (i, j) from the zone states along d: (4, 8), zones
        idx-2 .. idx+1, with PLM; (6, 8), zones idx-3 .. idx+2, with PPM."""
        nz = 6 if self.p.recon == PPM else 4
        q = np.ascontiguousarray(q4, dtype=np.float64).reshape(nz * NP)
        out = np.zeros(NU)
        cw = self.L.orc_face_flux_at(self.h, int(d), int(i), int(j), _p(q), _p(out))
        return out, cw

    def flags(self):
        out = np.zeros(self.shape, dtype=np.int32)
        self.L.orc_get_flags(self.h, _p(out, _I))
        return out

    def geom_table(self, kind=0):
        out = np.zeros((self.N[0], self.N[1], 34))
        self.L.orc_geom_table(self.h, kind, _p(out))
        return out

    def conn_table(self):
        out = np.zeros((self.N[0], self.N[1], 4, 4, 4))
        self.L.orc_conn_table(self.h, _p(out))
        return out

    def geom_at(self, X1, X2):
        g = Geom()
        self.L.orc_geom_at(self.h, X1, X2, C.byref(g))
        return g

    def conn_at(self, X1, X2):
        out = np.zeros((4, 4, 4))
        self.L.orc_conn_at(self.h, X1, X2, _p(out))
        return out

    def r_of_x1(self, X1):
        return self.L.orc_r_of_x1(self.h, X1)

    def th_of_x2(self, X2):
        return self.L.orc_th_of_x2(self.h, X2)

    def theta_at(self, X1, X2):
        """theta(X1, X2) with the polar cylindrification, and its partials
        (d theta/dX1, d theta/dX2)."""
        d = (C.c_double * 2)()
        th = self.L.orc_theta_at(self.h, X1, X2, d)
        return th, d[0], d[1]

    def x1_of_r(self, r):
        return self.L.orc_x1_of_r(self.h, r)

    def prim2cons(self, P, loc):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(NP, -1)
        loc = np.ascontiguousarray(loc, dtype=np.int32)
        n = P.shape[1]
        U = np.zeros((NU, n))
        self.L.orc_p2c_batch(self.h, _p(P), _p(loc, _I), _p(U), n)
        return U

    def con2prim(self, U, loc, guess, methods=15):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(NU, -1)
        guess = np.ascontiguousarray(guess, dtype=np.float64).reshape(NP, -1)
        loc = np.ascontiguousarray(loc, dtype=np.int32)
        n = U.shape[1]
        P = np.zeros((NP, n))
        flags = np.zeros(n, dtype=np.int32)
        iters = np.zeros(n, dtype=np.int32)
        self.L.orc_c2p_batch(self.h, _p(U), _p(loc, _I), _p(guess), _p(P), _p(flags, _I),
                             _p(iters, _I), n, methods)
        return P, flags, iters

    def con2prim_w(self, U, loc, guess, wguess, methods=15):
        """Inversion with an explicit Newton starting W per zone (<= 0: plain start)."""
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(NU, -1)
        guess = np.ascontiguousarray(guess, dtype=np.float64).reshape(NP, -1)
        wguess = np.ascontiguousarray(wguess, dtype=np.float64)
        loc = np.ascontiguousarray(loc, dtype=np.int32)
        n = U.shape[1]
        P = np.zeros((NP, n))
        flags = np.zeros(n, dtype=np.int32)
        iters = np.zeros(n, dtype=np.int32)
        self.L.orc_c2p_batch_w(self.h, _p(U), _p(loc, _I), _p(guess), _p(wguess), _p(P), _p(flags, _I),
                               _p(iters, _I), n, methods)
        return P, flags, iters

    def post_inversion(self, i, j, q, U):
        """Floors, magnetisation ceilings and Lorentz cap (Section 2.4) of
        active zone (i, j) after a successful inversion: (q', modified,
        ceiling hits, cap hits) from primitives q (8) and conserved U (9)."""
        q = np.array(q, dtype=np.float64).copy()
        U = np.array(U, dtype=np.float64).copy()
        out = np.zeros(3, dtype=np.int32)
        self.L.orc_post_inversion_at(self.h, int(i), int(j), _p(q), _p(U), _p(out, _I))
        return q, int(out[0]), int(out[1]), int(out[2])

    def mlp_samples(self, seed, first, n):
        """Samples first..first+n-1 of the seeded MLP training distribution:
        P (8, n), loc (n), U (9, n), features (5, n), labels log(W/D) (n)."""
        P = np.zeros((NP, n))
        loc = np.zeros(n, dtype=np.int32)
        U = np.zeros((NU, n))
        feat = np.zeros((5, n))
        lab = np.zeros(n)
        self.L.orc_mlp_samples(self.h, seed, first, n, _p(P), _p(loc, _I), _p(U), _p(feat), _p(lab))
        return P, loc, U, feat, lab


# ------------------------------------------------------------------ MLP helpers

MLP_NPARAM = 4609
MLP_SLICES = {"W1": (0, 320), "b1": (320, 384), "W2": (384, 4480), "b2": (4480, 4544),
              "W3": (4544, 4608), "b3": (4608, 4609)}


def bf16_round(x):
    """Round FP32 values to the nearest BF16 value (ties to even)."""
    L = lib()
    x = np.asarray(x, dtype=np.float32)
    return np.array([L.orc_bf16_round(float(v)) for v in x.ravel()], dtype=np.float32).reshape(x.shape)


def mlp_features(U, g: Geom):
    L = lib()
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.zeros(5)
    rc = L.orc_mlp_features(_p(U), C.byref(g), _p(f))
    return f, rc


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def mlp_forward(theta, norm, feat):
    """Predictions log(W/D) of features (5, n) with FP32 parameters theta."""
    theta, norm, feat = _f32(theta), _f32(norm), _f32(feat).reshape(5, -1)
    n = feat.shape[1]
    y = np.zeros(n)
    lib().orc_mlp_forward(_p(theta, _F), _p(norm, _F), _p(feat, _F), n, _p(y))
    return y


def mlp_loss_grad(theta, norm, feat, label):
    theta, norm, feat, label = _f32(theta), _f32(norm), _f32(feat).reshape(5, -1), _f32(label)
    n = feat.shape[1]
    g = np.zeros(MLP_NPARAM)
    loss = lib().orc_mlp_loss_grad(_p(theta, _F), _p(norm, _F), _p(feat, _F), _p(label, _F), n, _p(g))
    return loss, g


def mlp_loss_grad_exact(w, norm, feat, label):
    """Loss and gradient with FP64 weights w used unrounded."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    norm, feat, label = _f32(norm), _f32(feat).reshape(5, -1), _f32(label)
    n = feat.shape[1]
    g = np.zeros(MLP_NPARAM)
    loss = lib().orc_mlp_loss_grad_d(_p(w), _p(norm, _F), _p(feat, _F), _p(label, _F), n, _p(g))
    return loss, g


def mlp_adamw(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step in place on FP64 arrays theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    lib().orc_mlp_adamw(_p(theta), _p(m), _p(v), _p(grad), step, lr, beta1, beta2, eps, wd)


def mlp_train_steps(theta, norm, feat, label, batch, nsteps, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """nsteps of minibatch AdamW from theta (FP32); returns (theta, last loss)."""
    th = _f32(theta).copy()
    norm, feat, label = _f32(norm), _f32(feat).reshape(5, -1), _f32(label)
    n = feat.shape[1]
    fb = np.zeros((5, batch), dtype=np.float32)
    lb = np.zeros(batch, dtype=np.float32)
    work = np.zeros(4 * MLP_NPARAM)
    loss = lib().orc_mlp_train_steps(_p(th, _F), _p(norm, _F), _p(feat, _F), _p(label, _F), n, batch, nsteps,
                                     lr, beta1, beta2, eps, wd, _p(fb, _F), _p(lb, _F), _p(work))
    return th, loss


# ----------------------------------------------------------- pointwise helpers

def combine_dt(dtd):
    """Eq. 27: 1/dt = sum of 1/dt^l over the per-direction minima."""
    d = np.ascontiguousarray(dtd, dtype=np.float64)
    return lib().orc_combine_dt(_p(d))


def geom_from(gcov: np.ndarray) -> Geom:
    """Geometry record (gcon, sqrt(-g), alpha) for a 4x4 covariant metric."""
    L = lib()
    g = Geom()
    gc = np.ascontiguousarray(gcov, dtype=np.float64).reshape(16)
    inv = np.zeros(16)
    det = np.zeros(1)
    L.orc_invert4(_p(gc), _p(inv), _p(det))
    for a in range(16):
        g.gcov[a] = gc[a]
        g.gcon[a] = inv[a]
    g.gdet = float(np.sqrt(-det[0]))
    g.alpha = float(1.0 / np.sqrt(-inv[0]))
    return g


def state_of(q, g: Geom):
    L = lib()
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(18)
    L.orc_state_of(_p(q), C.byref(g), _p(out))
    return dict(ucon=out[0:4].copy(), ucov=out[4:8].copy(), bcon=out[8:12].copy(),
                bcov=out[12:16].copy(), bsq=out[16], gamma=out[17]), out


def prim_to_U(q, g: Geom, gam):
    L = lib()
    q = np.ascontiguousarray(q, dtype=np.float64)
    _, s = state_of(q, g)
    U = np.zeros(NU)
    L.orc_prim_to_U(_p(q), C.byref(g), _p(s), gam, _p(U))
    return U


def prim_to_F(q, g: Geom, gam, d):
    L = lib()
    q = np.ascontiguousarray(q, dtype=np.float64)
    _, s = state_of(q, g)
    F = np.zeros(NU)
    L.orc_prim_to_F(_p(q), C.byref(g), _p(s), gam, d, _p(F))
    return F


def wave_speeds(q, g: Geom, gam, d):
    L = lib()
    q = np.ascontiguousarray(q, dtype=np.float64)
    _, s = state_of(q, g)
    c1, c2 = C.c_double(), C.c_double()
    L.orc_wave_speeds(_p(q), C.byref(g), _p(s), gam, d, C.byref(c1), C.byref(c2))
    return c1.value, c2.value


def ppm_face(q6):
    """(left, right) PPM states at the face between q6[2] and q6[3]."""
    q = np.ascontiguousarray(q6, dtype=np.float64).reshape(6)
    out = np.zeros(2)
    lib().orc_ppm_face(_p(q), _p(out))
    return out[0], out[1]


def mc_slope(qm, q0, qp):
    return lib().orc_mc_slope(qm, q0, qp)


def ks_gcov(r, th, a):
    out = np.zeros(16)
    lib().orc_ks_gcov(r, th, a, _p(out))
    return out.reshape(4, 4)


def fm_ell(a, r_max):
    return lib().orc_fm_ell(a, r_max)


def fm_lnh(a, ell, r, th):
    return lib().orc_fm_lnh(a, ell, r, th)


def fm_ucon_bl(a, ell, r, th):
    out = np.zeros(4)
    lib().orc_fm_ucon_bl(a, ell, r, th, _p(out))
    return out


def uniform(seed, idx):
    return lib().orc_uniform(seed, idx)
