"""Thin ctypes binding of libfe.so (include/fe.h).

The functions below carry the C names and only marshal arguments: every
step of the computation runs in the CUDA kernels of libfe.so.  PyTorch is
used for device memory (torch tensors passed by pointer) and for the CUDA
stream.  Importing this module raises if libfe.so has not been built: there
is no CPU fallback.
"""
import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_uint64, c_void_p

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfe.so")

FE_OK = 0
FE_ERR_INVALID_ARG = -1
FE_ERR_CUDA = -2
FE_ERR_NOT_CONVERGED = -3
FE_ERR_NONFINITE = -4
FE_ERR_OOM = -5
FE_ERR_UNSUPPORTED = -6
FE_ERR_TOO_LARGE = -7
FE_NOALLOC_MAX_N = 64
FE_LES_MAX_M = 8
FE_PROFILE_MAX_KERNELS = 64

FE_FP64 = 0
FE_FP32_MIXED = 1
FE_BAROTROPIC = 0
FE_FOURIER = 1
FE_PCG_JACOBI = 0
FE_BICGSTAB_JACOBI = 1
FE_FCG_LEARNED = 2
FE_FGMRES_LEARNED = 3
FE_PCG_POLY = 4

FE_RHO, FE_UX, FE_UY, FE_UZ, FE_P, FE_T, FE_PHIX, FE_PHIY, FE_PHIZ, FE_Y0 = range(10)
FE_V0 = 17  # two-fluid dust: velocity component m of class j is FE_V0 + 3 j + m
FE_INIT_SPECTRAL = 0
FE_INIT_DERIVE = 1
FE_MAX_DUST = 8
FE_DUST_EQUILIBRIUM = 0
FE_DUST_TWO_FLUID = 1
FE_COUPLING_ONE_WAY = 0
FE_COUPLING_TWO_WAY = 1


class fe_params(ctypes.Structure):
    _fields_ = [("n_boxes", c_int32), ("N", POINTER(c_int32)), ("precision", c_int32), ("closure", c_int32),
                ("gamma", c_double), ("Pr", c_double), ("nu", POINTER(c_double)), ("n_dust", c_int32),
                ("tau_p", POINTER(c_double)), ("Y0", POINTER(c_double)), ("mach_rms", POINTER(c_double)),
                ("k0", POINTER(c_double)), ("seed", POINTER(c_uint64)), ("cfl", c_double),
                ("dt_growth_max", c_double), ("dt_max", c_double), ("n_corr", c_int32), ("solver", c_int32),
                ("p_tol", c_double), ("p_maxit", c_int32), ("transonic", c_int32), ("learned_every", c_int32),
                ("dust_model", c_int32), ("coupling", c_int32)]


class fe_step_info(ctypes.Structure):
    _fields_ = [("t", c_double), ("dt", c_double), ("iters", c_int32 * 4), ("rel_res", c_double * 4)]


class fe_solve_info(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("rel_res_true", c_double)]


class fe_diag(ctypes.Structure):
    _fields_ = [("ke", c_double), ("ke_u", c_double), ("enstrophy", c_double), ("taylor", c_double),
                ("rho_rms", c_double), ("mass", c_double), ("dust_mass", c_double * FE_MAX_DUST),
                ("energy", c_double), ("t", c_double), ("dt_prev", c_double)]


class fe_les_stats(ctypes.Structure):
    _fields_ = [("delta", c_double), ("k_sgs", c_double), ("pi_sgs", c_double), ("cs2_opt", c_double),
                ("corr", c_double), ("pi_model", c_double)]


class fe_profile_info(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("target_launches", ctypes.c_int64), ("target_ms", c_double),
                ("counts", ctypes.c_int64 * FE_PROFILE_MAX_KERNELS)]


EXPORTS = ["fe_create", "fe_init_state", "fe_set_field", "fe_get_field", "fe_set_fields", "fe_get_fields",
           "fe_set_clock", "fe_step",
           "fe_solve_pressure", "fe_diagnostics", "fe_q_criterion", "fe_profile_start", "fe_profile_stop",
           "fe_kernel_count", "fe_kernel_name", "fe_solve_pressure_noalloc", "fe_set_tiling", "fe_set_box_tiling", "fe_autotune",
           "fe_preconditioner_size", "fe_load_preconditioner", "fe_get_preconditioner", "fe_precond_apply",
           "fe_precond_train_step", "fe_precond_activation", "fe_harvest_pressure", "fe_use_graphs",
           "fe_use_plane_streaming", "fe_plane_streaming_active", "fe_precond_kernels", "fe_les_apriori", "fe_isosurface", "fe_raster_depth",
           "fe_destroy", "fe_strerror"]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libfe.so not found at %s: build it with paper_1404_0959_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    lib.fe_create.argtypes = [POINTER(fe_params), c_void_p, POINTER(c_void_p)]
    lib.fe_init_state.argtypes = [c_void_p, c_int, c_int]
    lib.fe_set_field.argtypes = [c_void_p, c_int, c_int, c_void_p, c_int]
    lib.fe_get_field.argtypes = [c_void_p, c_int, c_int, c_void_p, c_int]
    lib.fe_set_fields.argtypes = [c_void_p, c_int, c_int, POINTER(c_int), POINTER(c_void_p), c_int]
    lib.fe_get_fields.argtypes = [c_void_p, c_int, c_int, POINTER(c_int), POINTER(c_void_p), c_int]
    lib.fe_set_clock.argtypes = [c_void_p, c_int, c_double, c_double]
    lib.fe_step.argtypes = [c_void_p, c_int, POINTER(fe_step_info)]
    lib.fe_solve_pressure.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_double, c_double, c_int,
                                      POINTER(fe_solve_info)]
    lib.fe_diagnostics.argtypes = [c_void_p, c_int, POINTER(fe_diag), POINTER(c_double), c_int]
    lib.fe_q_criterion.argtypes = [c_void_p, c_int, c_void_p]
    lib.fe_profile_start.argtypes = [c_void_p, c_int]
    lib.fe_profile_stop.argtypes = [c_void_p, POINTER(fe_profile_info)]
    lib.fe_kernel_count.argtypes = []
    lib.fe_kernel_name.argtypes = [c_int]
    lib.fe_kernel_name.restype = ctypes.c_char_p
    lib.fe_solve_pressure_noalloc.argtypes = [c_int, c_void_p, c_void_p, c_void_p, c_double, c_double, c_int,
                                              c_void_p, POINTER(fe_solve_info)]
    lib.fe_preconditioner_size.argtypes = []
    lib.fe_preconditioner_size.restype = ctypes.c_long
    lib.fe_load_preconditioner.argtypes = [c_void_p, c_void_p, ctypes.c_size_t]
    lib.fe_get_preconditioner.argtypes = [c_void_p, c_void_p, ctypes.c_size_t, c_int]
    lib.fe_precond_apply.argtypes = [c_void_p, c_int, c_void_p, c_double, c_void_p]
    lib.fe_precond_train_step.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_double, c_double, POINTER(c_double)]
    lib.fe_precond_activation.argtypes = [c_void_p, c_int, c_void_p, ctypes.c_size_t]
    lib.fe_harvest_pressure.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_void_p), c_int, POINTER(c_int)]
    lib.fe_use_graphs.argtypes = [c_void_p, c_int]
    lib.fe_use_plane_streaming.argtypes = [c_void_p, c_int]
    lib.fe_plane_streaming_active.argtypes = [c_void_p]
    lib.fe_precond_kernels.argtypes = [c_void_p, c_int]
    lib.fe_les_apriori.argtypes = [c_void_p, c_int, c_int, c_double, POINTER(fe_les_stats), c_void_p]
    lib.fe_isosurface.argtypes = [c_void_p, c_int, c_void_p, c_double, c_void_p, ctypes.c_longlong,
                                  POINTER(ctypes.c_longlong), POINTER(c_double)]
    lib.fe_raster_depth.argtypes = [c_void_p, c_void_p, ctypes.c_longlong, c_int, c_double, c_void_p]
    lib.fe_set_tiling.argtypes = [c_void_p, c_int]
    lib.fe_set_box_tiling.argtypes = [c_void_p, c_int, c_int]
    lib.fe_autotune.argtypes = [c_void_p, c_int, POINTER(c_int)]
    lib.fe_destroy.argtypes = [c_void_p]
    lib.fe_destroy.restype = None
    lib.fe_strerror.argtypes = [c_int]
    lib.fe_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("fe_destroy", "fe_strerror", "fe_kernel_name", "fe_preconditioner_size"):
            getattr(lib, name).restype = c_int
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class FeError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, lib().fe_strerror(code).decode(), code))


def _check(code, where):
    if code != FE_OK:
        raise FeError(code, where)
    return code


# ---- C entry points (same names, marshalling only) -------------------------------------------
def fe_create(params, stream=None):
    ctx = c_void_p()
    _check(lib().fe_create(byref(params), c_void_p(stream or 0), byref(ctx)), "fe_create")
    return ctx


def fe_init_state(ctx, box, mode):
    return _check(lib().fe_init_state(ctx, box, mode), "fe_init_state")


def fe_set_field(ctx, box, field, ptr, is_device):
    return _check(lib().fe_set_field(ctx, box, field, c_void_p(ptr), int(is_device)), "fe_set_field")


def fe_get_field(ctx, box, field, ptr, is_device):
    return _check(lib().fe_get_field(ctx, box, field, c_void_p(ptr), int(is_device)), "fe_get_field")


def _field_arrays(fields, ptrs):
    n = len(fields)
    if len(ptrs) != n:
        raise ValueError("one pointer per field")
    return n, (c_int * n)(*fields), (c_void_p * n)(*[c_void_p(p) for p in ptrs])


def fe_set_fields(ctx, box, fields, ptrs, is_device):
    n, f, p = _field_arrays(fields, ptrs)
    return _check(lib().fe_set_fields(ctx, box, n, f, p, int(is_device)), "fe_set_fields")


def fe_get_fields(ctx, box, fields, ptrs, is_device):
    n, f, p = _field_arrays(fields, ptrs)
    return _check(lib().fe_get_fields(ctx, box, n, f, p, int(is_device)), "fe_get_fields")


def fe_set_clock(ctx, box, t, dt_prev):
    return _check(lib().fe_set_clock(ctx, box, t, dt_prev), "fe_set_clock")


def fe_step(ctx, nsteps, info=None):
    """Returns the raw status (FE_ERR_NOT_CONVERGED / NONFINITE are reported, not raised)."""
    code = lib().fe_step(ctx, nsteps, info)
    if code not in (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_NONFINITE):
        raise FeError(code, "fe_step")
    return code


def fe_solve_pressure(ctx, box, b_ptr, x_ptr, dt, tol, maxit):
    info = fe_solve_info()
    code = lib().fe_solve_pressure(ctx, box, c_void_p(b_ptr), c_void_p(x_ptr), dt, tol, maxit, byref(info))
    if code not in (FE_OK, FE_ERR_NOT_CONVERGED):
        raise FeError(code, "fe_solve_pressure")
    return code, info


def fe_diagnostics(ctx, box, nbins=0):
    d = fe_diag()
    spec = (c_double * max(nbins, 1))()
    _check(lib().fe_diagnostics(ctx, box, byref(d), spec if nbins > 0 else None, nbins), "fe_diagnostics")
    return d, np.array(spec[:nbins])


def fe_q_criterion(ctx, box, q_ptr):
    return _check(lib().fe_q_criterion(ctx, box, c_void_p(q_ptr)), "fe_q_criterion")


def fe_profile_start(ctx, kernel_id=-1):
    return _check(lib().fe_profile_start(ctx, kernel_id), "fe_profile_start")


def fe_profile_stop(ctx):
    info = fe_profile_info()
    _check(lib().fe_profile_stop(ctx, byref(info)), "fe_profile_stop")
    return info


def fe_kernel_count():
    return lib().fe_kernel_count()


def fe_kernel_name(kernel_id):
    return lib().fe_kernel_name(kernel_id).decode()


def kernel_id(name):
    for k in range(fe_kernel_count()):
        if fe_kernel_name(k) == name:
            return k
    raise KeyError(name)


def fe_solve_pressure_noalloc(N, psi_ptr, b_ptr, x_ptr, dt, tol, maxit, stream=None):
    """Allocation-free FP64 pressure solve (for callers that cannot allocate device memory)."""
    info = fe_solve_info()
    code = lib().fe_solve_pressure_noalloc(N, c_void_p(psi_ptr), c_void_p(b_ptr), c_void_p(x_ptr), dt, tol, maxit,
                                           c_void_p(stream or 0), byref(info))
    if code not in (FE_OK, FE_ERR_NOT_CONVERGED):
        raise FeError(code, "fe_solve_pressure_noalloc")
    return code, info


def fe_preconditioner_size():
    return int(lib().fe_preconditioner_size())


def fe_load_preconditioner(ctx, weights):
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).reshape(-1))
    return _check(lib().fe_load_preconditioner(ctx, w.ctypes.data, w.size), "fe_load_preconditioner")


def fe_get_preconditioner(ctx, gradients=False):
    w = np.empty(fe_preconditioner_size(), dtype=np.float32)
    _check(lib().fe_get_preconditioner(ctx, w.ctypes.data, w.size, int(gradients)), "fe_get_preconditioner")
    return w


def fe_les_apriori(ctx, box, m, cs, fields_ptr=None):
    """A-priori LES statistics of a box (dict); fields_ptr: optional device array of 10 N^3 values."""
    out = fe_les_stats()
    _check(lib().fe_les_apriori(ctx, box, m, cs, byref(out), c_void_p(fields_ptr) if fields_ptr else None),
           "fe_les_apriori")
    return {k: getattr(out, k) for k, _ in fe_les_stats._fields_}


def fe_isosurface(ctx, box, field_ptr, iso, tri_ptr=None, max_tri=0):
    """(total triangle count, total area); the first max_tri triangles go to tri_ptr (9 doubles each)."""
    n = ctypes.c_longlong(0)
    a = c_double(0.0)
    _check(lib().fe_isosurface(ctx, box, c_void_p(field_ptr), iso, c_void_p(tri_ptr) if tri_ptr else None, max_tri,
                               byref(n), byref(a)), "fe_isosurface")
    return n.value, a.value


def fe_raster_depth(ctx, tri_ptr, ntri, width, extent, depth_ptr):
    return _check(lib().fe_raster_depth(ctx, c_void_p(tri_ptr) if tri_ptr else None, ntri, width, extent,
                                        c_void_p(depth_ptr)), "fe_raster_depth")


def fe_precond_apply(ctx, box, r_ptr, dt, z_ptr):
    return _check(lib().fe_precond_apply(ctx, box, c_void_p(r_ptr), dt, c_void_p(z_ptr)), "fe_precond_apply")


def fe_precond_train_step(ctx, box, r_ptr, e_ptr, dt, lr):
    loss = c_double(0.0)
    _check(lib().fe_precond_train_step(ctx, box, c_void_p(r_ptr), c_void_p(e_ptr), dt, lr, byref(loss)),
           "fe_precond_train_step")
    return loss.value


def fe_precond_activation(ctx, layer, count):
    out = np.empty(count, dtype=np.float32)
    _check(lib().fe_precond_activation(ctx, layer, out.ctypes.data, count), "fe_precond_activation")
    return out


def fe_harvest_pressure(ctx, b_ptrs, x_ptrs):
    n = len(b_ptrs)
    bb = (c_void_p * n)(*[c_void_p(p) for p in b_ptrs])
    xx = (c_void_p * n)(*[c_void_p(p) for p in x_ptrs])
    got = c_int(0)
    code = lib().fe_harvest_pressure(ctx, bb, xx, n, byref(got))
    if code not in (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_NONFINITE):
        raise FeError(code, "fe_harvest_pressure")
    return code, got.value


def fe_use_graphs(ctx, on=True):
    return _check(lib().fe_use_graphs(ctx, int(bool(on))), "fe_use_graphs")


def fe_precond_kernels(ctx, mode):
    return _check(lib().fe_precond_kernels(ctx, int(mode)), "fe_precond_kernels")


def fe_use_plane_streaming(ctx, on=True):
    return _check(lib().fe_use_plane_streaming(ctx, int(bool(on))), "fe_use_plane_streaming")


def fe_plane_streaming_active(ctx):
    code = lib().fe_plane_streaming_active(ctx)
    if code < 0:
        raise FeError(code, "fe_plane_streaming_active")
    return bool(code)


def fe_set_tiling(ctx, tz):
    return _check(lib().fe_set_tiling(ctx, tz), "fe_set_tiling")


def fe_set_box_tiling(ctx, box, tz):
    return _check(lib().fe_set_box_tiling(ctx, box, tz), "fe_set_box_tiling")


def fe_autotune(ctx, trials=2):
    best = c_int(0)
    _check(lib().fe_autotune(ctx, trials, byref(best)), "fe_autotune")
    return best.value


def fe_destroy(ctx):
    lib().fe_destroy(ctx)


def fe_strerror(code):
    return lib().fe_strerror(code).decode()


# ---- convenience wrapper ------------------------------------------------------------------------
class Solver:
    """A context plus the host arrays its parameters point to.

    boxes: list of dicts with keys N, nu, tau_p (list), Y0 (list), mach_rms, k0, seed.
    Fields are exchanged as torch tensors on the device (or numpy on the host).
    """

    def __init__(self, boxes, precision=FE_FP64, closure=FE_BAROTROPIC, gamma=1.4, Pr=0.7, cfl=0.5,
                 dt_growth_max=1.2, dt_max=float("inf"), n_corr=2, solver=FE_PCG_JACOBI, p_tol=1e-10,
                 p_maxit=500, transonic=False, learned_every=1, stream=None, dust_model=FE_DUST_EQUILIBRIUM,
                 coupling=FE_COUPLING_ONE_WAY):
        import torch
        self.torch = torch
        nb = len(boxes)
        nd = len(boxes[0].get("tau_p", []))
        self.nd = nd
        self.boxes = boxes
        self.precision = precision
        self.dtype = torch.float64 if precision == FE_FP64 else torch.float32
        self.np_dtype = np.float64 if precision == FE_FP64 else np.float32
        self._N = (c_int32 * nb)(*[b["N"] for b in boxes])
        self._nu = (c_double * nb)(*[b.get("nu", 0.005) for b in boxes])
        self._mach = (c_double * nb)(*[b.get("mach_rms", 0.2) for b in boxes])
        self._k0 = (c_double * nb)(*[b.get("k0", 4.0) for b in boxes])
        self._seed = (c_uint64 * nb)(*[b.get("seed", 0) for b in boxes])
        tp = [v for b in boxes for v in b.get("tau_p", [])]
        y0 = [v for b in boxes for v in b.get("Y0", [])]
        self._tau = (c_double * max(len(tp), 1))(*tp)
        self._y0 = (c_double * max(len(y0), 1))(*y0)
        self.params = fe_params(nb, self._N, precision, closure, gamma, Pr, self._nu, nd, self._tau, self._y0,
                                self._mach, self._k0, self._seed, cfl, dt_growth_max,
                                dt_max if np.isfinite(dt_max) else 0.0, n_corr, solver, p_tol, p_maxit,
                                int(bool(transonic)), int(learned_every), int(dust_model), int(coupling))
        self.two_fluid = dust_model == FE_DUST_TWO_FLUID
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.ctx = fe_create(self.params, stream)
        self.n_corr = n_corr

    def close(self):
        if getattr(self, "ctx", None) is not None:
            fe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def N(self, box=0):
        return self.boxes[box]["N"]

    def init_state(self, box=-1, mode=FE_INIT_SPECTRAL):
        fe_init_state(self.ctx, box, mode)

    def set_field(self, box, field, value):
        t = self.torch
        N = self.N(box)
        if isinstance(value, t.Tensor) and value.is_cuda:
            v = value.to(self.dtype).contiguous().reshape(N, N, N)
            fe_set_field(self.ctx, box, field, v.data_ptr(), 1)
        else:
            v = np.ascontiguousarray(np.asarray(value, dtype=self.np_dtype).reshape(N, N, N))
            fe_set_field(self.ctx, box, field, v.ctypes.data, 0)

    def get_field(self, box, field, device=False):
        N = self.N(box)
        if device:
            out = self.torch.empty((N, N, N), dtype=self.dtype, device="cuda")
            fe_get_field(self.ctx, box, field, out.data_ptr(), 1)
            return out
        out = np.empty((N, N, N), dtype=self.np_dtype)
        fe_get_field(self.ctx, box, field, out.ctypes.data, 0)
        return out

    def set_state(self, box, rho, u, Y, T=None, V=None):
        """rho, u, Y (and T), then p and phi derived; two-fluid dust velocities V[j][m] (u unless given)."""
        self.set_field(box, FE_RHO, rho)
        for d in range(3):
            self.set_field(box, FE_UX + d, u[d])
        for j, y in enumerate(Y):
            self.set_field(box, FE_Y0 + j, y)
        if T is not None:
            self.set_field(box, FE_T, T)
        self.init_state(box, FE_INIT_DERIVE)
        if V is not None:
            for j, vj in enumerate(V):
                for m in range(3):
                    self.set_field(box, FE_V0 + 3 * j + m, vj[m])

    def load_state(self, box, st, t=0.0, dt_prev=0.0):
        """Set every state field (rho, u, phi, p, Y, T) as given, then the clock (checkpoint restore)."""
        self.set_field(box, FE_RHO, st["rho"])
        for d in range(3):
            self.set_field(box, FE_UX + d, st["u"][d])
            self.set_field(box, FE_PHIX + d, st["phi"][d])
        self.set_field(box, FE_P, st["p"])
        for j, y in enumerate(st["Y"]):
            self.set_field(box, FE_Y0 + j, y)
        if st.get("T") is not None:
            self.set_field(box, FE_T, st["T"])
        if st.get("V") is not None:
            for j, vj in enumerate(st["V"]):
                for m in range(3):
                    self.set_field(box, FE_V0 + 3 * j + m, vj[m])
        fe_set_clock(self.ctx, box, t, dt_prev)

    def get_state(self, box=0):
        g = self.get_field
        st = {"rho": g(box, FE_RHO), "u": [g(box, FE_UX + d) for d in range(3)],
              "phi": [g(box, FE_PHIX + d) for d in range(3)], "p": g(box, FE_P),
              "Y": [g(box, FE_Y0 + j) for j in range(self.nd)]}
        st["T"] = g(box, FE_T) if self.params.closure == FE_FOURIER else None
        if self.two_fluid:
            st["V"] = [[g(box, FE_V0 + 3 * j + m) for m in range(3)] for j in range(self.nd)]
        return st

    def step(self, nsteps=1):
        nb = self.params.n_boxes
        info = (fe_step_info * nb)()
        code = fe_step(self.ctx, nsteps, info)
        return code, [dict(t=i.t, dt=i.dt, iters=list(i.iters)[:self.n_corr],
                           rel_res=list(i.rel_res)[:self.n_corr]) for i in info]

    def solve_pressure(self, box, b, dt, tol, maxit):
        t = self.torch
        b = b.to(self.dtype).contiguous()
        x = t.empty_like(b)
        code, info = fe_solve_pressure(self.ctx, box, b.data_ptr(), x.data_ptr(), dt, tol, maxit)
        return code, x, info

    def diagnostics(self, box=0, nbins=0):
        d, spec = fe_diagnostics(self.ctx, box, nbins)
        out = {k: getattr(d, k) for k in ("ke", "ke_u", "enstrophy", "taylor", "rho_rms", "mass", "energy", "t",
                                          "dt_prev")}
        out["dust_mass"] = list(d.dust_mass)[:self.nd]
        if nbins > 0:
            out["spectrum"] = spec
        return out

    def use_graphs(self, on=True):
        fe_use_graphs(self.ctx, on)

    def use_plane_streaming(self, on=True):
        fe_use_plane_streaming(self.ctx, on)

    def plane_streaming_active(self):
        return fe_plane_streaming_active(self.ctx)

    def autotune(self, trials=2):
        return fe_autotune(self.ctx, trials)

    def set_tiling(self, tz):
        fe_set_tiling(self.ctx, tz)

    def set_box_tiling(self, box, tz):
        fe_set_box_tiling(self.ctx, box, tz)

    def profile_start(self, kernel=None):
        fe_profile_start(self.ctx, -1 if kernel is None else kernel_id(kernel))

    def profile_stop(self):
        info = fe_profile_stop(self.ctx)
        n = min(fe_kernel_count(), FE_PROFILE_MAX_KERNELS)
        return dict(launches=info.launches, target_launches=info.target_launches, target_ms=info.target_ms,
                    counts={fe_kernel_name(k): info.counts[k] for k in range(n) if info.counts[k]})

    def q_criterion(self, box=0):
        N = self.N(box)
        q = self.torch.empty((N, N, N), dtype=self.dtype, device="cuda")
        fe_q_criterion(self.ctx, box, q.data_ptr())
        return q
