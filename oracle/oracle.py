"""ctypes wrapper around the C oracle (fcd_oracle.c).

Test infrastructure only. Builds the C file with gcc on first use into
oracle/_build/ and exposes numpy-array entry points. Each wrapper names the
paper passage its C routine follows.
"""
import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "fcd_oracle.c")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 9
DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int)


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("rho", C.c_double * 3), ("nu", C.c_double * 3), ("chi", C.c_double * 3),
        ("mobility", C.c_double), ("xi", C.c_double), ("eta", C.c_double),
        ("Ca", C.c_double), ("Bo_m", C.c_double), ("alpha", C.c_double),
        ("r1", C.c_double), ("r2", C.c_double), ("xc", C.c_double), ("yc", C.c_double),
        ("s13_over_s12", C.c_double), ("s23_over_s12", C.c_double),
        ("sigma23", C.c_double), ("u_max", C.c_double),
        ("ferro_phase", C.c_int),
        ("mag_tol", C.c_double), ("mag_max_iter", C.c_int),
        ("eps_n", C.c_double),
        ("open_x", C.c_int),
    ]


class Derived(C.Structure):
    _fields_ = [
        ("u_avg", C.c_double), ("sigma", (C.c_double * 3) * 3), ("gamma", C.c_double * 3),
        ("gammaT", C.c_double), ("tau", C.c_double * 3), ("tau_phi", C.c_double),
        ("mu0H0sq", C.c_double), ("H0", C.c_double), ("G", C.c_double),
    ]


class Track(C.Structure):
    _fields_ = [("b_step", C.c_long), ("bx", C.c_int), ("by", C.c_int)]


class Obs(C.Structure):
    _fields_ = [
        ("step", C.c_long), ("t_star", C.c_double),
        ("T_o", C.c_double), ("T_i", C.c_double), ("lx_o", C.c_double), ("ly_o", C.c_double),
        ("lx_i", C.c_double), ("ly_i", C.c_double),
        ("xc_core", C.c_double), ("yc_core", C.c_double),
        ("xc_shell", C.c_double), ("yc_shell", C.c_double),
        ("mass", C.c_double * 3),
        ("breakup", C.c_int), ("b_step", C.c_long), ("xb", C.c_double), ("yb", C.c_double),
        ("tb_star", C.c_double), ("Lb_star", C.c_double), ("yb_star", C.c_double),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "mass" else v
        return d


def build(force=False):
    """Compile fcd_oracle.c with gcc (FP contraction off so x86 and Arm agree)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fcd_oracle.h"))):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC]
        try:  # row-parallel node loops when the compiler has OpenMP
            subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_tables.argtypes = [DP, IP, IP, DP, DP]
        L.orc_derive.argtypes = [C.POINTER(Params), C.POINTER(Derived)]
        L.orc_gamma.argtypes = [C.c_double, C.c_double, DP]
        L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, DP]
        L.orc_mrt_apply.argtypes = [DP, C.c_double, DP]
        L.orc_dH.argtypes = [C.POINTER(Derived), C.c_double, DP, DP]
        L.orc_H.argtypes = [C.POINTER(Derived), C.c_double, DP]
        L.orc_H.restype = C.c_double
        L.orc_chem.argtypes = [C.POINTER(Derived), C.c_double, C.c_double, DP, DP, DP]
        L.orc_grad.argtypes = [C.c_int, C.c_int, DP, DP, DP]
        L.orc_lap.argtypes = [C.c_int, C.c_int, DP, DP]
        L.orc_phase.argtypes = [C.POINTER(Params), DP, DP, DP]
        L.orc_mag_apply.argtypes = [C.c_int, C.c_int, DP, DP, C.c_double, C.c_double, DP]
        L.orc_mag_rhs.argtypes = [C.c_int, C.c_int, DP, C.c_double, C.c_double, DP]
        L.orc_mag_solve.argtypes = [C.c_int, C.c_int, DP, C.c_double, C.c_double, DP,
                                    C.c_double, C.c_int, IP, DP]
        L.orc_mag_solve.restype = C.c_int
        L.orc_forces.argtypes = [C.POINTER(Params), DP, DP, DP, DP]
        L.orc_init.argtypes = [C.POINTER(Params), DP, DP, DP, DP, IP, DP]
        L.orc_init.restype = C.c_int
        L.orc_step.argtypes = [C.POINTER(Params), DP, DP, DP, DP, C.c_long, C.c_long,
                               C.POINTER(Track), IP, DP]
        L.orc_step.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = C.c_int
        L.orc_observe.argtypes = [C.POINTER(Params), DP, C.POINTER(Track), C.c_long,
                                  C.POINTER(Obs)]
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(DP)


def make_params(cfg):
    """Fill the oracle's own parameter struct from a workload dict."""
    p = Params()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    for i in range(3):
        p.rho[i] = cfg["rho"][i]
        p.nu[i] = cfg["nu"][i]
        p.chi[i] = cfg["chi"][i]
    p.mobility = cfg.get("mobility", 0.3)
    p.xi = cfg.get("xi", 5.0)
    p.eta = cfg.get("eta", 0.0)
    p.Ca = cfg.get("Ca", 0.1)
    p.Bo_m = cfg.get("Bo_m", 0.0)
    p.alpha = cfg.get("alpha", 0.0)
    p.r1, p.r2 = cfg["r1"], cfg["r2"]
    p.xc, p.yc = cfg["xc"], cfg["yc"]
    p.s13_over_s12 = cfg.get("s13_over_s12", 1.0)
    p.s23_over_s12 = cfg.get("s23_over_s12", 1.0)
    p.sigma23 = cfg.get("sigma23", 0.0)
    p.u_max = cfg.get("u_max", 0.01)
    p.ferro_phase = int(cfg.get("ferro_phase", 0))
    p.mag_tol = cfg.get("mag_tol", 1e-10)
    p.mag_max_iter = int(cfg.get("mag_max_iter", 100000))
    p.eps_n = cfg.get("eps_n", 1e-12)
    p.open_x = int(cfg.get("open_x", 0))
    return p


def tables():
    w = np.zeros(Q)
    ex = np.zeros(Q, np.int32)
    ey = np.zeros(Q, np.int32)
    M = np.zeros(Q * Q)
    Mi = np.zeros(Q * Q)
    lib().orc_tables(_p(w), ex.ctypes.data_as(IP), ey.ctypes.data_as(IP), _p(M), _p(Mi))
    return w, ex, ey, M.reshape(Q, Q), Mi.reshape(Q, Q)


def derive(cfg):
    d = Derived()
    p = make_params(cfg)
    lib().orc_derive(C.byref(p), C.byref(d))
    return d


def gamma(ux, uy):
    out = np.zeros(Q)
    lib().orc_gamma(ux, uy, _p(out))
    return out


def feq(pstar, ux, uy):
    out = np.zeros(Q)
    lib().orc_feq(pstar, ux, uy, _p(out))
    return out


def mrt_apply(h, s_nu):
    h = np.ascontiguousarray(h, dtype=np.float64)
    out = np.zeros(Q)
    lib().orc_mrt_apply(_p(h), s_nu, _p(out))
    return out


def free_energy(cfg, phi3, eta=None):
    d = derive(cfg)
    ph = np.ascontiguousarray(phi3, dtype=np.float64)
    e = cfg.get("eta", 0.0) if eta is None else eta
    return lib().orc_H(C.byref(d), e, _p(ph))


def dH(cfg, phi3, eta=None):
    d = derive(cfg)
    ph = np.ascontiguousarray(phi3, dtype=np.float64)
    out = np.zeros(3)
    e = cfg.get("eta", 0.0) if eta is None else eta
    lib().orc_dH(C.byref(d), e, _p(ph), _p(out))
    return out


def chem(cfg, phi3, lap3):
    d = derive(cfg)
    ph = np.ascontiguousarray(phi3, dtype=np.float64)
    lp = np.ascontiguousarray(lap3, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_chem(C.byref(d), cfg.get("eta", 0.0), cfg.get("xi", 5.0), _p(ph), _p(lp), _p(out))
    return out


def grad(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    ny, nx = a.shape
    gx, gy = np.zeros_like(a), np.zeros_like(a)
    lib().orc_grad(nx, ny, _p(a), _p(gx), _p(gy))
    return gx, gy


def lap(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    ny, nx = a.shape
    out = np.zeros_like(a)
    lib().orc_lap(nx, ny, _p(a), _p(out))
    return out


def phase(cfg, g):
    p = make_params(cfg)
    N = p.nx * p.ny
    phi = np.zeros((3, p.ny, p.nx))
    k = np.zeros((p.ny, p.nx))
    assert g.size == 2 * Q * N
    lib().orc_phase(C.byref(p), _p(g), _p(phi), _p(k))
    return phi, k


def mag_apply(k, psi, H0, alpha):
    k = np.ascontiguousarray(k, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ny, nx = k.shape
    out = np.zeros_like(k)
    lib().orc_mag_apply(nx, ny, _p(k), _p(psi), H0, alpha, _p(out))
    return out


def mag_rhs(k, H0, alpha):
    k = np.ascontiguousarray(k, dtype=np.float64)
    ny, nx = k.shape
    out = np.zeros_like(k)
    lib().orc_mag_rhs(nx, ny, _p(k), H0, alpha, _p(out))
    return out


def mag_solve(k, H0, alpha, psi=None, tol=1e-13, max_iter=100000):
    k = np.ascontiguousarray(k, dtype=np.float64)
    ny, nx = k.shape
    psi = np.zeros_like(k) if psi is None else np.ascontiguousarray(psi, dtype=np.float64).copy()
    it = C.c_int(0)
    res = C.c_double(0)
    st = lib().orc_mag_solve(nx, ny, _p(k), H0, alpha, _p(psi), tol, max_iter, C.byref(it),
                             C.byref(res))
    return psi, st, it.value, res.value


FORCE_NAMES = ["Fs_x", "Fs_y", "Fm_x", "Fm_y", "Fp_x", "Fp_y", "Fmu_x", "Fmu_y",
               "ux", "uy", "rho", "pstar", "Hx", "Hy"]


def forces(cfg, f, g, psi):
    p = make_params(cfg)
    out = np.zeros((14, p.ny, p.nx))
    lib().orc_forces(C.byref(p), _p(f), _p(g), _p(np.ascontiguousarray(psi)), _p(out))
    return dict(zip(FORCE_NAMES, out))


class Sim:
    """Whole-path oracle run: state arrays plus the sticky breakup record."""

    def __init__(self, cfg):
        self.cfg = dict(cfg)
        self.p = make_params(cfg)
        nx, ny = self.p.nx, self.p.ny
        self.f = np.zeros((Q, ny, nx))
        self.g = np.zeros((2, Q, ny, nx))
        self.psi = np.zeros((ny, nx))
        self.macro = np.zeros((3, ny, nx))
        self.track = Track(-1, 0, 0)
        self.step_count = 0
        it = C.c_int(0)
        res = C.c_double(0)
        self.status = lib().orc_init(C.byref(self.p), _p(self.f), _p(self.g), _p(self.psi),
                                     _p(self.macro), C.byref(it), C.byref(res))
        self.mag_iters, self.mag_resid = it.value, res.value

    def step(self, n=1):
        it = C.c_int(0)
        res = C.c_double(0)
        st = lib().orc_step(C.byref(self.p), _p(self.f), _p(self.g), _p(self.psi),
                            _p(self.macro), self.step_count, n, C.byref(self.track),
                            C.byref(it), C.byref(res))
        self.step_count += n
        self.mag_iters, self.mag_resid = it.value, res.value
        self.status = st
        return st

    def phi(self):
        return phase(self.cfg, self.g)[0]

    def observe(self):
        o = Obs()
        lib().orc_observe(C.byref(self.p), _p(self.g), C.byref(self.track), self.step_count,
                          C.byref(o))
        return o.as_dict()

    def derived(self):
        return derive(self.cfg)


def set_threads(n):
    """Threads of the oracle's row-parallel node loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def max_threads():
    """Host processors usable by the oracle (1 when built without OpenMP)."""
    return lib().orc_max_threads()


def deg(a):
    return a * math.pi / 180.0
