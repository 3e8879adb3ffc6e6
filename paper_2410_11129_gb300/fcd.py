"""Thin ctypes binding of libfcd.so (C ABI in include/fcd.h).

Argument marshalling only: every step of the path runs in the CUDA library.
The functions keep the C names; ``Channel`` wraps one context for Python use
(PyTorch supplies the CUDA stream and, optionally, the device allocator).
Loading fails loudly when the library is missing; there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

DP = C.POINTER(C.c_double)

FCD_OK, FCD_EINVAL, FCD_ENOMEM, FCD_ECUDA, FCD_ENOCONV, FCD_EUNSTABLE, FCD_ESTATE = range(7)
FCD_FP64, FCD_FP32, FCD_FP32_OFFSET = range(3)
PRECISION = {"fp64": FCD_FP64, "fp32": FCD_FP32, "fp32_offset": FCD_FP32_OFFSET}
FIELDS = {"phi1": 0, "phi2": 1, "phi3": 2, "ux": 3, "uy": 4, "pstar": 5, "psi": 6}
STATUS = {0: "FCD_OK", 1: "FCD_EINVAL", 2: "FCD_ENOMEM", 3: "FCD_ECUDA", 4: "FCD_ENOCONV",
          5: "FCD_EUNSTABLE", 6: "FCD_ESTATE"}


class fcd_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("rho", C.c_double * 3), ("nu", C.c_double * 3), ("chi", C.c_double * 3),
        ("mobility", C.c_double), ("xi", C.c_double), ("eta", C.c_double),
        ("Ca", C.c_double), ("Bo_m", C.c_double), ("alpha", C.c_double),
        ("r1", C.c_double), ("r2", C.c_double), ("xc", C.c_double), ("yc", C.c_double),
        ("s13_over_s12", C.c_double), ("s23_over_s12", C.c_double), ("sigma23", C.c_double),
        ("u_max", C.c_double), ("ferro_phase", C.c_int), ("precision", C.c_int),
        ("mag_tol", C.c_double), ("mag_max_iter", C.c_int), ("eps_n", C.c_double),
        ("open_x", C.c_int),
    ]


class fcd_obs(C.Structure):
    _fields_ = [
        ("step", C.c_long), ("t_star", C.c_double),
        ("T_o", C.c_double), ("T_i", C.c_double),
        ("lx_o", C.c_double), ("ly_o", C.c_double), ("lx_i", C.c_double), ("ly_i", C.c_double),
        ("xc_core", C.c_double), ("yc_core", C.c_double),
        ("xc_shell", C.c_double), ("yc_shell", C.c_double),
        ("mass", C.c_double * 3),
        ("breakup", C.c_int), ("b_step", C.c_long), ("xb", C.c_double), ("yb", C.c_double),
        ("tb_star", C.c_double), ("Lb_star", C.c_double), ("yb_star", C.c_double),
        ("mag_iters", C.c_int), ("mag_resid", C.c_double),
    ]

    def as_dict(self):
        return {n: (list(getattr(self, n)) if n == "mass" else getattr(self, n))
                for n, _ in self._fields_}


DIRECTIONS = ("Bo_m", "Ca", "alpha", "nu_r")  # order of the tangent directions


class fcd_tangent_obs(C.Structure):
    _fields_ = [
        ("step", C.c_long), ("T_o", C.c_double), ("overlap", C.c_double),
        ("lx_o", C.c_double), ("ly_o", C.c_double),
        ("dT_o", C.c_double * 4), ("doverlap", C.c_double * 4),
        ("dlx_o", C.c_double * 4), ("dly_o", C.c_double * 4),
    ]

    def as_dict(self):
        return {n: (list(getattr(self, n)) if n[0] == "d" else getattr(self, n))
                for n, _ in self._fields_}


class fcd_adjoint_out(C.Structure):
    _fields_ = [
        ("step", C.c_long), ("T_o", C.c_double), ("overlap", C.c_double), ("J", C.c_double),
        ("grad", C.c_double * 4), ("capped_solves", C.c_long), ("recomputed_steps", C.c_long),
        ("solve_cycles", C.c_longlong),
    ]

    def as_dict(self):
        return {n: (list(getattr(self, n)) if n == "grad" else getattr(self, n))
                for n, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None

# symbol -> (restype, argtypes)
_SIGS = {
    "fcd_set_allocator": (None, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "fcd_create": (C.c_int, [C.POINTER(fcd_params), C.POINTER(C.c_void_p)]),
    "fcd_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fcd_step": (C.c_int, [C.c_void_p, C.c_long]),
    "fcd_solve_magnetic": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int), DP]),
    "fcd_observables": (C.c_int, [C.c_void_p, C.POINTER(fcd_obs)]),
    "fcd_get_field": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "fcd_get_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fcd_set_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]),
    "fcd_state_bytes": (C.c_size_t, [C.c_void_p]),
    "fcd_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fcd_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fcd_get_derived": (C.c_int, [C.c_void_p, DP]),
    "fcd_derive_params": (C.c_int, [C.POINTER(fcd_params), DP]),
    "fcd_kernel_launches": (C.c_long, [C.c_void_p]),
    "fcd_solver_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "fcd_collide_tile_height": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "fcd_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "fcd_last_step_profile": (C.c_int, [C.c_void_p, DP]),
    "fcd_last_error": (C.c_char_p, [C.c_void_p]),
    "fcd_observe_populations_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int,
                                                   C.c_void_p, C.POINTER(fcd_obs)]),
    "fcd_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "fcd_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fcd_batch_step": (C.c_int, [C.c_void_p, C.c_long]),
    "fcd_batch_observables": (C.c_int, [C.c_void_p, C.POINTER(fcd_obs)]),
    "fcd_batch_size": (C.c_int, [C.c_void_p]),
    "fcd_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "fcd_batch_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    "fcd_batch_instance": (C.c_void_p, [C.c_void_p, C.c_int]),
    "fcd_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "fcd_batch_destroy": (None, [C.c_void_p]),
    "fcd_create_tangent": (C.c_int, [C.POINTER(fcd_params), C.POINTER(C.c_void_p)]),
    "fcd_tangent_observables": (C.c_int, [C.c_void_p, C.POINTER(fcd_tangent_obs)]),
    "fcd_create_adjoint": (C.c_int, [C.POINTER(fcd_params), C.c_int, C.POINTER(C.c_void_p)]),
    "fcd_adjoint_gradient": (C.c_int, [C.c_void_p, C.c_double, C.c_double,
                                       C.POINTER(fcd_adjoint_out), C.c_void_p, C.c_void_p]),
    "fcd_adjoint_gradient_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.POINTER(fcd_adjoint_out), C.c_void_p, C.c_void_p]),
    "fcd_destroy": (None, [C.c_void_p]),
}


def lib_path():
    return _build.LIB


def load(build=True):
    """Load libfcd.so (building it first when asked); raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libfcd.so is missing at %s; run the build first" % path)
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FcdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def make_params(cfg):
    """fcd_params from a workload dictionary (see workloads.py)."""
    p = fcd_params()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    for i in range(3):
        p.rho[i], p.nu[i], p.chi[i] = cfg["rho"][i], cfg["nu"][i], cfg["chi"][i]
    p.mobility = cfg.get("mobility", 0.3)
    p.xi = cfg.get("xi", 5.0)
    p.eta = cfg.get("eta", 0.0)
    p.Ca = cfg.get("Ca", 0.1)
    p.Bo_m = cfg.get("Bo_m", 0.0)
    p.alpha = cfg.get("alpha", 0.0)
    p.r1, p.r2, p.xc, p.yc = cfg["r1"], cfg["r2"], cfg["xc"], cfg["yc"]
    p.s13_over_s12 = cfg.get("s13_over_s12", 1.0)
    p.s23_over_s12 = cfg.get("s23_over_s12", 1.0)
    p.sigma23 = cfg.get("sigma23", 0.0)
    p.u_max = cfg.get("u_max", 0.01)
    p.ferro_phase = int(cfg.get("ferro_phase", 0))
    prec = cfg.get("precision", "fp64")
    p.precision = PRECISION[prec] if isinstance(prec, str) else int(prec)
    p.mag_tol = cfg.get("mag_tol", 1e-10)
    p.mag_max_iter = int(cfg.get("mag_max_iter", 200))
    p.eps_n = cfg.get("eps_n", 1e-12 if p.precision == FCD_FP64 else 1e-6)
    p.open_x = int(cfg.get("open_x", 0))
    return p


DERIVED = ["u_avg", "sigma12", "sigma13", "sigma23", "gamma1", "gamma2", "gamma3", "gammaT",
           "tau1", "tau2", "tau3", "tau_phi", "mu0H0sq", "H0", "G"]


def derive_params(cfg):
    """The library's lattice mapping of a workload (fcd_derive_params): host
    code only, no context and no GPU."""
    L = load()
    p = make_params(cfg)
    out = (C.c_double * 15)()
    st = L.fcd_derive_params(C.byref(p), out)
    if st != FCD_OK:
        raise FcdError(st, L.fcd_last_error(None).decode())
    return dict(zip(DERIVED, list(out)))


_torch_alloc = None


def use_torch_allocator():
    """Route later fcd_create allocations through PyTorch's caching allocator."""
    global _torch_alloc
    import torch

    def _alloc(size, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(size)))
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    _torch_alloc = (ALLOC_FN(_alloc), FREE_FN(_free))
    load().fcd_set_allocator(_torch_alloc[0], _torch_alloc[1], None)


class Channel:
    """One context of the coupled step (owns the C handle)."""

    _create = "fcd_create"

    def __init__(self, cfg, stream=None, torch_alloc=True):
        L = load()
        self.cfg = dict(cfg)
        if torch_alloc and _torch_alloc is None:
            use_torch_allocator()
        self.params = make_params(cfg)
        h = C.c_void_p()
        st = self._make(L, h)
        if st != FCD_OK:
            raise FcdError(st, L.fcd_last_error(None).decode())
        self.h = h
        self.nx, self.ny = self.params.nx, self.params.ny
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.check(L.fcd_set_stream(self.h, C.c_void_p(stream)))

    def _make(self, L, h):
        return getattr(L, self._create)(C.byref(self.params), C.byref(h))

    def check(self, st, allow=()):
        if st != FCD_OK and st not in allow:
            raise FcdError(st, load().fcd_last_error(self.h).decode())
        return st

    def step(self, n=1):
        return self.check(load().fcd_step(self.h, int(n)))

    def solve_magnetic(self, tol=0.0, max_iter=0):
        it, res = C.c_int(0), C.c_double(0)
        st = load().fcd_solve_magnetic(self.h, tol, max_iter, C.byref(it), C.byref(res))
        self.check(st, allow=(FCD_ENOCONV,))
        return it.value, res.value, st

    def observe(self, allow=()):
        o = fcd_obs()
        st = load().fcd_observables(self.h, C.byref(o))
        self.check(st, allow=allow)
        return o.as_dict()

    def field(self, name, out=None):
        N = self.nx * self.ny
        if out is None:
            out = np.empty((self.ny, self.nx))
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else int(out.data_ptr())
        self.check(load().fcd_get_field(self.h, FIELDS[name], C.c_void_p(ptr), N))
        return out

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((2, 9, self.ny, self.nx))
        psi = np.empty((self.ny, self.nx))
        self.check(load().fcd_get_populations(self.h, C.c_void_p(f.ctypes.data),
                                              C.c_void_p(g.ctypes.data), C.c_void_p(psi.ctypes.data)))
        return f, g, psi

    def set_populations(self, f=None, g=None, psi=None, step=0):
        ptr = lambda a: None if a is None else C.c_void_p(np.ascontiguousarray(a, np.float64).ctypes.data)
        keep = [np.ascontiguousarray(a, np.float64) if a is not None else None for a in (f, g, psi)]
        self.check(load().fcd_set_populations(self.h, *[ptr(a) for a in keep], int(step)))

    def state_bytes(self):
        return load().fcd_state_bytes(self.h)

    def get_state(self, buf):
        """buf: writable host numpy uint8 array or torch tensor (host or device)."""
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else int(buf.data_ptr())
        n = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        return self.check(load().fcd_get_state(self.h, C.c_void_p(ptr), n))

    def set_state(self, buf):
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else int(buf.data_ptr())
        n = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        return self.check(load().fcd_set_state(self.h, C.c_void_p(ptr), n))

    def derived(self):
        out = (C.c_double * 15)()
        self.check(load().fcd_get_derived(self.h, out))
        return dict(zip(DERIVED, list(out)))

    def solver_stats(self):
        out = (C.c_longlong * 5)()
        self.check(load().fcd_solver_stats(self.h, out))
        return dict(zip(["heads", "vcycles", "twogrid", "sweeps", "capped"], list(out)))

    def collide_tile_height(self):
        """Rows per tile of the collide-stream kernel (FP32: timed at create)."""
        out = C.c_int(0)
        self.check(load().fcd_collide_tile_height(self.h, C.byref(out)))
        return out.value

    def set_profiling(self, on=True):
        self.check(load().fcd_set_profiling(self.h, 1 if on else 0))

    def last_step_profile(self):
        ms = (C.c_double * 4)()
        self.check(load().fcd_last_step_profile(self.h, ms))
        return dict(zip(["phase", "solve", "collide", "step"], list(ms)))

    def kernel_launches(self):
        return load().fcd_kernel_launches(self.h)

    def close(self):
        if getattr(self, "h", None):
            load().fcd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tangent(Channel):
    """FP64 context that also carries the derivatives of its state along
    (Bo_m, Ca, alpha, nu_r) (fcd_create_tangent)."""

    _create = "fcd_create_tangent"

    def tangent_observe(self, allow=()):
        o = fcd_tangent_obs()
        st = load().fcd_tangent_observables(self.h, C.byref(o))
        self.check(st, allow=allow)
        return o.as_dict()


class Adjoint(Channel):
    """FP64 periodic context that keeps a checkpoint every `checkpoint` steps;
    its reverse sweep gives dJ/d(Bo_m, Ca, alpha, nu_r) and dJ/d(initial
    populations) for J = w_T T_o + w_overlap overlap (fcd_create_adjoint)."""

    def __init__(self, cfg, checkpoint=500, stream=None, torch_alloc=True):
        self.checkpoint = int(checkpoint)
        super().__init__(cfg, stream, torch_alloc)

    def _make(self, L, h):
        return L.fcd_create_adjoint(C.byref(self.params), self.checkpoint, C.byref(h))

    def gradient(self, w_T=1.0, w_overlap=0.0, initial=False, allow=()):
        """Reverse sweep back to step 0. With initial=True the result also holds
        df0 (9, ny, nx) and dg0 (2, 9, ny, nx): dJ/d(populations at step 0)."""
        o = fcd_adjoint_out()
        df0 = dg0 = None
        if initial:
            df0 = np.empty((9, self.ny, self.nx))
            dg0 = np.empty((2, 9, self.ny, self.nx))
        ptr = lambda a: None if a is None else C.c_void_p(a.ctypes.data)
        st = load().fcd_adjoint_gradient(self.h, float(w_T), float(w_overlap), C.byref(o),
                                         ptr(df0), ptr(dg0))
        self.check(st, allow=allow)
        out = o.as_dict()
        if initial:
            out["df0"], out["dg0"] = df0, dg0
        return out

    def gradient_state(self, seed_f=None, seed_g=None, initial=False, allow=()):
        """Reverse sweep for any functional J of the final state, given as
        seed_f = dJ/df (9, ny, nx) and/or seed_g = dJ/dg (2, 9, ny, nx)."""
        o = fcd_adjoint_out()
        df0 = dg0 = None
        if initial:
            df0 = np.empty((9, self.ny, self.nx))
            dg0 = np.empty((2, 9, self.ny, self.nx))
        keep = [None if a is None else np.ascontiguousarray(a, np.float64) for a in (seed_f, seed_g)]
        ptr = lambda a: None if a is None else C.c_void_p(a.ctypes.data)
        st = load().fcd_adjoint_gradient_state(self.h, ptr(keep[0]), ptr(keep[1]), C.byref(o),
                                               ptr(df0), ptr(dg0))
        self.check(st, allow=allow)
        out = o.as_dict()
        if initial:
            out["df0"], out["dg0"] = df0, dg0
        return out

    def values(self):
        """(T_o, overlap) of the current state (no sweep: J = 0 has zero gradient)."""
        o = self.gradient(0.0, 0.0, allow=(FCD_ENOCONV,))
        return o["T_o"], o["overlap"]


def with_parameters(cfg, theta):
    """cfg with (Bo_m, Ca, alpha [rad], nu_r) set; nu_r = nu_3 / nu_2 (Eq. 39)."""
    bo, ca, al, nr = (float(v) for v in theta)
    out = dict(cfg)
    out["Bo_m"], out["Ca"], out["alpha"] = bo, ca, al
    nu = list(cfg["nu"])
    nu[1] = nu[2] / nr
    out["nu"] = nu
    return out


def parameters_of(cfg):
    return (cfg["Bo_m"], cfg["Ca"], cfg["alpha"], cfg["nu"][2] / cfg["nu"][1])


def _droplet_function():
    import torch

    class DropletObservables(torch.autograd.Function):
        """(T_o, overlap) of cfg after `steps` coupled steps, as a function of
        theta = (Bo_m, Ca, alpha, nu_r). Forward runs the tangent-linear
        context; backward applies the 2 x 4 Jacobian it produced."""

        @staticmethod
        def forward(ctx, theta, cfg, steps):
            ch = Tangent(with_parameters(cfg, theta.detach().cpu().tolist()))
            try:
                if steps:
                    ch.step(int(steps))
                o = ch.tangent_observe()
            finally:
                ch.close()
            J = torch.tensor([o["dT_o"], o["doverlap"]], dtype=torch.float64)
            ctx.save_for_backward(J)
            return torch.tensor([o["T_o"], o["overlap"]], dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (J,) = ctx.saved_tensors
            g = grad_out.detach().to(device="cpu", dtype=torch.float64) @ J
            return g.to(device=grad_out.device), None, None

    return DropletObservables


def _droplet_adjoint_function():
    import torch

    class DropletObservablesAdjoint(torch.autograd.Function):
        """(T_o, overlap) of cfg after `steps` coupled steps, as a function of
        theta = (Bo_m, Ca, alpha, nu_r). Forward runs the plain FP64 step with
        checkpoints; backward runs the discrete adjoint once, for the scalar
        grad_out . (T_o, overlap)."""

        @staticmethod
        def forward(ctx, theta, cfg, steps, checkpoint):
            ch = Adjoint(with_parameters(cfg, theta.detach().cpu().tolist()), checkpoint)
            try:
                if steps:
                    ch.step(int(steps))
                vals = ch.values()
            except Exception:
                ch.close()
                raise
            ctx.ch = ch
            return torch.tensor(vals, dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            w = grad_out.detach().to(device="cpu", dtype=torch.float64).tolist()
            ch = ctx.ch
            try:
                o = ch.gradient(w[0], w[1])
            finally:
                ch.close()
                ctx.ch = None
            g = torch.tensor(o["grad"], dtype=torch.float64, device=grad_out.device)
            return g, None, None, None

    return DropletObservablesAdjoint


def _final_state_function():
    import torch

    class FinalState(torch.autograd.Function):
        """The populations (f, g) after `steps` coupled steps, as a function of
        theta = (Bo_m, Ca, alpha, nu_r): forward runs the plain FP64 step with
        checkpoints, backward runs one discrete-adjoint sweep seeded with the
        incoming gradients of f and g."""

        @staticmethod
        def forward(ctx, theta, cfg, steps, checkpoint):
            ch = Adjoint(with_parameters(cfg, theta.detach().cpu().tolist()), checkpoint)
            try:
                if steps:
                    ch.step(int(steps))
                f, g, _ = ch.populations()
            except Exception:
                ch.close()
                raise
            ctx.ch = ch
            ctx.theta_device = theta.device
            return torch.from_numpy(f), torch.from_numpy(g)

        @staticmethod
        def backward(ctx, grad_f, grad_g):
            ch = ctx.ch
            as_np = lambda x: None if x is None else x.detach().cpu().numpy()
            try:
                o = ch.gradient_state(as_np(grad_f), as_np(grad_g))
            finally:
                ch.close()
                ctx.ch = None
            return (torch.tensor(o["grad"], dtype=torch.float64, device=ctx.theta_device),
                    None, None, None)

    return FinalState


_FINAL_STATE_FN = None


def final_state(theta, cfg, steps, checkpoint=500):
    """Differentiable final populations (f (9, ny, nx), g (2, 9, ny, nx), FP64,
    on the host): any torch loss of them back-propagates to theta through one
    reverse sweep of the discrete adjoint."""
    global _FINAL_STATE_FN
    if _FINAL_STATE_FN is None:
        _FINAL_STATE_FN = _final_state_function()
    return _FINAL_STATE_FN.apply(theta, cfg, steps, checkpoint)


_DROPLET_FN = None
_DROPLET_ADJ_FN = None


def droplet_observables(theta, cfg, steps, method="tangent", checkpoint=500):
    """Differentiable (T_o, overlap): torch.autograd entry point of the tangent
    form (method="tangent": the 2 x 4 Jacobian is formed in forward) or of the
    discrete adjoint (method="adjoint": one reverse sweep in backward)."""
    global _DROPLET_FN, _DROPLET_ADJ_FN
    if method == "tangent":
        if _DROPLET_FN is None:
            _DROPLET_FN = _droplet_function()
        return _DROPLET_FN.apply(theta, cfg, steps)
    if method == "adjoint":
        if _DROPLET_ADJ_FN is None:
            _DROPLET_ADJ_FN = _droplet_adjoint_function()
        return _DROPLET_ADJ_FN.apply(theta, cfg, steps, checkpoint)
    raise ValueError("method must be 'tangent' or 'adjoint'")


class _Instance(Channel):
    """A context owned by a Batch (not destroyed on its own)."""

    def __init__(self, handle, cfg):
        self.h = C.c_void_p(handle)
        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.nx, self.ny = self.params.nx, self.params.ny

    def close(self):
        self.h = None


class Batch:
    """Many independent channels advanced together (fcd_batch_*)."""

    def __init__(self, cfgs, stream=None, torch_alloc=True):
        L = load()
        if torch_alloc and _torch_alloc is None:
            use_torch_allocator()
        self.cfgs = [dict(c) for c in cfgs]
        arr = (fcd_params * len(cfgs))(*[make_params(c) for c in cfgs])
        h = C.c_void_p()
        st = L.fcd_batch_create(arr, len(cfgs), C.byref(h))
        if st != FCD_OK:
            raise FcdError(st, L.fcd_batch_last_error(None).decode())
        self.h = h
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        L.fcd_batch_set_stream(self.h, C.c_void_p(stream))
        self.instances = [_Instance(L.fcd_batch_instance(self.h, i), c) for i, c in enumerate(cfgs)]

    def step(self, n=1):
        st = load().fcd_batch_step(self.h, int(n))
        if st != FCD_OK:
            raise FcdError(st, load().fcd_batch_last_error(self.h).decode())

    def observe(self, allow=()):
        out = (fcd_obs * len(self.cfgs))()
        st = load().fcd_batch_observables(self.h, out)
        if st != FCD_OK and st not in allow:
            raise FcdError(st, load().fcd_batch_last_error(self.h).decode())
        return [o.as_dict() for o in out]

    def tuning(self):
        """{"mode": 1 batched kernels, 0 instance streams, -1 still timing;
        "batched": instances on the batched kernels; "groups"; "tile_h": the
        collide tile height per group}."""
        md, nb, ng, th = C.c_int(0), C.c_int(0), C.c_int(0), (C.c_int * 64)()
        load().fcd_batch_tuning(self.h, C.byref(md), C.byref(nb), C.byref(ng), th, 64)
        return {"mode": md.value, "batched": nb.value, "groups": ng.value,
                "tile_h": list(th)[:ng.value]}

    def set_mode(self, mode):
        """1: batched kernels, 0: every instance on its own stream, -1: time both again."""
        st = load().fcd_batch_set_mode(self.h, int(mode))
        if st != FCD_OK:
            raise FcdError(st, load().fcd_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            load().fcd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# C-name aliases (same names as the ABI)
def fcd_create(cfg):
    return Channel(cfg)


def fcd_step(ch, n):
    return ch.step(n)


def fcd_solve_magnetic(ch, tol=0.0, max_iter=0):
    return ch.solve_magnetic(tol, max_iter)


def fcd_observables(ch):
    return ch.observe()


def fcd_destroy(ch):
    ch.close()
