"""ctypes binding of libflups (include/flups.h): argument marshalling only.

Every step of the projection runs in the library's CUDA kernels; this module only turns
torch CUDA tensors (or raw integer device addresses) into pointers, passes the current
CUDA stream, and raises on a non-OK status.  There is no CPU fallback: if libflups.so is
missing or cannot be loaded, every call raises.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflups.so")

OK, EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, ENONFINITE, ENOCONV, ESTATE, ETIMEOUT = range(9)
BC = {"periodic": 0, "walls": 1}
XY_BC = {"periodic": 0, "neumann": 1, "dirichlet": 2, "neumann_dirichlet": 3, "dirichlet_neumann": 4}
PREC = {"fp64": 0, "fp32_refine": 1}
HIST = 16

# every entry point declared in include/flups.h
SYMBOLS = [
    "flups_plan_create", "flups_plan_destroy", "flups_set_stream", "flups_workspace_bytes", "flups_launch_count",
    "flups_set_density", "flups_get_rho0", "flups_rhs", "flups_solve", "flups_correct",
    "flups_project_host", "flups_status_string", "flups_solve_fp64_noalloc",
    "flups_set_profiling", "flups_profile_read", "flups_kernel_name",
    "flups_solve_graphable", "flups_solve_result",
    "flups_batch_create", "flups_batch_solve", "flups_batch_destroy", "flups_batch_graph_kernels",
    "flups_batch_member_tuning", "flups_last_cuda_error", "flups_varcoef_solve",
    "flups_pnet_create", "flups_pnet_destroy", "flups_pnet_set_params", "flups_pnet_get_params",
    "flups_pnet_get_grads", "flups_pnet_get_adam", "flups_pnet_set_adam", "flups_pnet_predict", "flups_pnet_train_step", "flups_pnet_eval_loss",
    "flups_pnet_launch_count", "flups_pnet_set_profiling", "flups_pnet_profile_read", "flups_pnet_kernel_name",
    "flups_selftest_wait_timeout", "flups_momentum_predict", "flups_plan_create_bc", "flups_plan_sync",
    "flups_solve_host", "flups_vof_step",
]
PNET_NKERNELS = 6
PNET_NPARAMS = 15601
NKERNELS = 26
MOM_PAIR = 0
MOM_FP64 = 1


class FlupsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        extra = ""
        if status in (ECUDA, ENOMEM):
            extra = f" ({lib().flups_last_cuda_error().decode()})"
        super().__init__(f"{where}: {status_string(status)}{extra}")


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("rel_res_hist", ctypes.c_double * HIST)]

    def history(self):
        return [h for h in self.rel_res_hist[: max(self.iters, 0)]]


_lib = None


def lib():
    """Load libflups.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2204_08834_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.flups_plan_create.argtypes = [ctypes.POINTER(P), I, I, I, D, D, ctypes.POINTER(D), I, I, V]
        L.flups_plan_create_bc.argtypes = [ctypes.POINTER(P), I, I, I, D, D, ctypes.POINTER(D), I, I, I, I, V]
        L.flups_plan_destroy.argtypes = [P]
        L.flups_set_stream.argtypes = [P, V]
        L.flups_workspace_bytes.argtypes = [P]
        L.flups_workspace_bytes.restype = ctypes.c_size_t
        L.flups_launch_count.argtypes = [P]
        L.flups_launch_count.restype = ctypes.c_ulonglong
        L.flups_set_density.argtypes = [P, V, D]
        L.flups_get_rho0.argtypes = [P, ctypes.POINTER(D)]
        L.flups_plan_sync.argtypes = [P]
        L.flups_rhs.argtypes = [P, V, V, V, V, V, D, D, D, V]
        L.flups_solve.argtypes = [P, V, V, D, I, ctypes.POINTER(Info)]
        L.flups_correct.argtypes = [P, V, V, V, D, D, D, V, V, V]
        L.flups_project_host.argtypes = [P, V, V, V, V, V, V, D, D, D, D, I, V, ctypes.POINTER(Info)]
        L.flups_solve_host.argtypes = [P, V, V, D, I, ctypes.POINTER(Info)]
        L.flups_vof_step.argtypes = [P, V, V, V, V, D, D, V]
        L.flups_solve_fp64_noalloc.argtypes = [I, I, I, D, D, ctypes.POINTER(D), I, V, V, V]
        L.flups_set_profiling.argtypes = [P, I]
        L.flups_profile_read.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)]
        L.flups_solve_graphable.argtypes = [P, V, V, D, I]
        L.flups_solve_result.argtypes = [P, D, ctypes.POINTER(Info)]
        IP = ctypes.POINTER(ctypes.c_int)
        DP = ctypes.POINTER(ctypes.c_double)
        L.flups_batch_create.argtypes = [ctypes.POINTER(P), I, IP, IP, IP, DP, DP, ctypes.POINTER(DP), IP, I, I, V]
        L.flups_batch_solve.argtypes = [P, ctypes.POINTER(V), ctypes.POINTER(V), D, I, ctypes.POINTER(Info)]
        L.flups_batch_destroy.argtypes = [P]
        L.flups_batch_graph_kernels.argtypes = [P]
        L.flups_batch_graph_kernels.restype = ctypes.c_ulonglong
        L.flups_batch_member_tuning.argtypes = [P, I, IP, IP]
        L.flups_varcoef_solve.argtypes = [P, V, V, V, D, I, ctypes.POINTER(Info)]
        L.flups_momentum_predict.argtypes = [P, V, V, V, V, V, V, V, D, D, D, D, D, D, I]
        FP = ctypes.POINTER(ctypes.c_float)
        L.flups_pnet_create.argtypes = [ctypes.POINTER(P), I, I, I, FP, V]
        L.flups_pnet_destroy.argtypes = [P]
        L.flups_pnet_set_params.argtypes = [P, FP]
        L.flups_pnet_get_params.argtypes = [P, FP]
        L.flups_pnet_get_grads.argtypes = [P, FP]
        L.flups_pnet_get_adam.argtypes = [P, FP, FP, ctypes.POINTER(ctypes.c_longlong)]
        L.flups_pnet_set_adam.argtypes = [P, FP, FP, ctypes.c_longlong]
        L.flups_pnet_predict.argtypes = [P, V, D, V, V, V]
        L.flups_pnet_train_step.argtypes = [P, V, D, V, V, V, ctypes.c_float, DP]
        L.flups_pnet_eval_loss.argtypes = [P, V, D, V, V, V, DP]
        L.flups_pnet_launch_count.argtypes = [P]
        L.flups_pnet_launch_count.restype = ctypes.c_ulonglong
        L.flups_pnet_set_profiling.argtypes = [P, I]
        L.flups_pnet_profile_read.argtypes = [P, DP, ctypes.POINTER(ctypes.c_longlong)]
        L.flups_pnet_kernel_name.argtypes = [I]
        L.flups_pnet_kernel_name.restype = ctypes.c_char_p
        L.flups_selftest_wait_timeout.argtypes = [V, I]
        L.flups_last_cuda_error.argtypes = []
        L.flups_last_cuda_error.restype = ctypes.c_char_p
        L.flups_kernel_name.argtypes = [I]
        L.flups_kernel_name.restype = ctypes.c_char_p
        L.flups_status_string.argtypes = [I]
        L.flups_status_string.restype = ctypes.c_char_p
        for name in SYMBOLS:
            if name not in ("flups_status_string", "flups_workspace_bytes", "flups_launch_count",
                            "flups_kernel_name", "flups_batch_graph_kernels", "flups_last_cuda_error",
                            "flups_pnet_launch_count", "flups_pnet_kernel_name"):
                getattr(L, name).restype = I
        _lib = L
    return _lib


def status_string(s):
    return lib().flups_status_string(int(s)).decode()


def _check(status, where):
    if status != OK:
        raise FlupsError(status, where)


def ptr(x):
    """Device address of a contiguous float64 CUDA tensor, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda or x.dtype.__repr__() != "torch.float64" or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 CUDA tensor")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def ptr32(x):
    """Device address of a contiguous float32 CUDA tensor (or an int address)."""
    if isinstance(x, int):
        return x
    if not (hasattr(x, "data_ptr") and x.is_cuda and x.dtype.__repr__() == "torch.float32" and x.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return x.data_ptr()


def momentum_state(nz, ny, nx, device="cuda"):
    """Zeroed M state for Plan.momentum_predict: [3][nz][ny][nx] pairs (hi, lo) of float32."""
    import torch
    return torch.zeros((3, nz, ny, nx, 2), dtype=torch.float32, device=device)


def hptr(a):
    """Host address of a C-contiguous float64 numpy array."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data


def current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Plan:
    """One projection plan (flups_plan_create).  Fields are [nz][ny][nx] float64."""

    def __init__(self, nx, ny, nz, dx, dy, dzf, bc="periodic", prec="fp32_refine", stream=None, bcx="periodic",
                 bcy="periodic"):
        self.shape = (nz, ny, nx)
        self.bc, self.prec, self.bcx, self.bcy = bc, prec, bcx, bcy
        dz = np.ascontiguousarray(np.broadcast_to(np.asarray(dzf, dtype=np.float64), (nz,)))
        self._dz = dz
        h = ctypes.c_void_p()
        st = lib().flups_plan_create_bc(ctypes.byref(h), int(nx), int(ny), int(nz), float(dx), float(dy),
                                        dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), XY_BC[bcx], XY_BC[bcy],
                                        BC[bc], PREC[prec], stream)
        _check(st, "flups_plan_create_bc")
        self._h = h

    @classmethod
    def for_case(cls, case, prec="fp32_refine", stream=None):
        nz, ny, nx = case.shape
        if stream is None:
            stream = current_stream()
        return cls(nx, ny, nz, case.dx, case.dy, case.dzf, case.bc, prec, stream)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().flups_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def launches(self):
        return lib().flups_launch_count(self._h)

    @property
    def workspace_bytes(self):
        return lib().flups_workspace_bytes(self._h)

    def set_profiling(self, on=True):
        _check(lib().flups_set_profiling(self._h, int(bool(on))), "flups_set_profiling")

    def profile(self):
        """{kernel name: (total ms, timed regions)} recorded since the last call (synchronises)."""
        ms = (ctypes.c_double * NKERNELS)()
        n = (ctypes.c_longlong * NKERNELS)()
        _check(lib().flups_profile_read(self._h, ms, n), "flups_profile_read")
        return {lib().flups_kernel_name(k).decode(): (ms[k], n[k]) for k in range(NKERNELS) if n[k]}

    def set_stream(self, stream):
        _check(lib().flups_set_stream(self._h, stream), "flups_set_stream")

    def set_density(self, rho, rho0=0.0):
        _check(lib().flups_set_density(self._h, ptr(rho), float(rho0)), "flups_set_density")

    def rho0(self):
        r = ctypes.c_double()
        _check(lib().flups_get_rho0(self._h, ctypes.byref(r)), "flups_get_rho0")
        return r.value

    def sync(self, check=True):
        """Wait for the plan's stream; raise on (or, with check=False, return) a latched device error."""
        st = lib().flups_plan_sync(self._h)
        if check:
            _check(st, "flups_plan_sync")
        return st

    def rhs(self, u, v, w, pn, pnm1, c1, c2, dt, f):
        _check(lib().flups_rhs(self._h, ptr(u), ptr(v), ptr(w), ptr(pn), ptr(pnm1), float(c1), float(c2),
                               float(dt), ptr(f)), "flups_rhs")

    def solve(self, f, p, rtol=1e-10, max_iter=16, info=True, check=True):
        inf = Info() if info else None
        st = lib().flups_solve(self._h, ptr(f), ptr(p), float(rtol), int(max_iter),
                               ctypes.byref(inf) if inf is not None else None)
        if check:
            _check(st, "flups_solve")
        return inf if check else (st, inf)

    def solve_graphable(self, f, p, rtol=1e-10, max_iter=4):
        _check(lib().flups_solve_graphable(self._h, ptr(f), ptr(p), float(rtol), int(max_iter)),
               "flups_solve_graphable")

    def solve_result(self, rtol=1e-10, check=True):
        inf = Info()
        st = lib().flups_solve_result(self._h, float(rtol), ctypes.byref(inf))
        if check:
            _check(st, "flups_solve_result")
        return inf if check else (st, inf)

    def correct(self, p, pn, pnm1, c1, c2, dt, u, v, w):
        _check(lib().flups_correct(self._h, ptr(p), ptr(pn), ptr(pnm1), float(c1), float(c2), float(dt),
                                   ptr(u), ptr(v), ptr(w)), "flups_correct")

    def varcoef_solve(self, rho, f, p, rtol=1e-12, max_iter=500, check=True):
        """Exact variable-coefficient pressure D((rho0/rho_f) G p) = f - <f> (PCG)."""
        inf = Info()
        st = lib().flups_varcoef_solve(self._h, ptr(rho), ptr(f), ptr(p), float(rtol), int(max_iter),
                                       ctypes.byref(inf))
        if check:
            _check(st, "flups_varcoef_solve")
        return inf if check else (st, inf)

    def momentum_predict(self, u, v, w, us, vs, ws, m_state, nu, g, dt, dt_prev, arith=MOM_PAIR):
        """u** = u^n + dt (f1 M^n - f2 M^{n-1} + g) (Sec. 3.3, Eq. uss_predic); m_state (see
        momentum_state) holds M^{n-1} on entry (read when dt_prev > 0) and M^n on return."""
        st = lib().flups_momentum_predict(self._h, ptr(u), ptr(v), ptr(w), ptr(us), ptr(vs), ptr(ws), ptr32(m_state),
                                          float(nu), float(g[0]), float(g[1]), float(g[2]), float(dt),
                                          float(dt_prev), int(arith))
        _check(st, "flups_momentum_predict")

    def project_host(self, u, v, w, rho, pn, pnm1, c1, c2, dt, p_out, rtol=1e-10, max_iter=16):
        """Whole projection on HOST numpy arrays (u, v, w updated in place; p_out written)."""
        inf = Info()
        st = lib().flups_project_host(self._h, hptr(u), hptr(v), hptr(w), hptr(rho), hptr(pn),
                                      hptr(pnm1) if pnm1 is not None else None, float(c1), float(c2),
                                      float(dt), float(rtol), int(max_iter), hptr(p_out), ctypes.byref(inf))
        _check(st, "flups_project_host")
        return inf

    def vof_step(self, phi, u, v, w, dt, beta=2.0, stages=None):
        """One VoF step (flups_vof_step): phi (DEVICE float64) updated in place."""
        _check(lib().flups_vof_step(self._h, ptr(phi), ptr(u), ptr(v), ptr(w), float(dt), float(beta),
                                    ptr(stages) if stages is not None else None), "flups_vof_step")

    def solve_host(self, f, p_out, rtol=1e-10, max_iter=16, check=True):
        """flups_solve on HOST numpy arrays f (read) and p_out (written)."""
        inf = Info()
        st = lib().flups_solve_host(self._h, hptr(f), hptr(p_out), float(rtol), int(max_iter), ctypes.byref(inf))
        if check:
            _check(st, "flups_solve_host")
        return inf


def selftest_wait_timeout(limit=4096, stream=None):
    """Status of flups_selftest_wait_timeout (ETIMEOUT when the bounded wait works)."""
    if stream is None:
        stream = current_stream()
    return lib().flups_selftest_wait_timeout(stream, int(limit))


def solve_fp64_noalloc(nx, ny, nz, dx, dy, dzf, bc, f, p, stream=None, check=True):
    """FP64 direct solve without any device allocation (flups_solve_fp64_noalloc).

    For callers that may not call cudaMalloc (the library then uses one fixed 16 MiB
    device array per GPU as workspace); calls that overlap on the GPU race on that array.
    """
    dz = np.ascontiguousarray(np.broadcast_to(np.asarray(dzf, dtype=np.float64), (nz,)))
    if stream is None:
        stream = current_stream()
    st = lib().flups_solve_fp64_noalloc(int(nx), int(ny), int(nz), float(dx), float(dy),
                                        dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), BC[bc], ptr(f),
                                        ptr(p), stream)
    if check:
        _check(st, "flups_solve_fp64_noalloc")
    return st


class Batch:
    """Ensemble of independent FP32-refine solves in one CUDA graph launch (flups_batch_*).

    members: sequence of (nx, ny, nz, dx, dy, dzf, bc) with dzf a scalar or nz widths.
    """

    def __init__(self, members, nstreams=8, autotune=True, stream=None):
        n = len(members)
        self.n = n
        self.shapes = [(m[2], m[1], m[0]) for m in members]
        ci = ctypes.c_int * n
        cd = ctypes.c_double * n
        self._dz = [np.ascontiguousarray(np.broadcast_to(np.asarray(m[5], dtype=np.float64), (m[2],)))
                    for m in members]
        dzp = (ctypes.POINTER(ctypes.c_double) * n)(*[d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                                      for d in self._dz])
        if stream is None:
            stream = current_stream()
        h = ctypes.c_void_p()
        st = lib().flups_batch_create(ctypes.byref(h), n, ci(*[m[0] for m in members]), ci(*[m[1] for m in members]),
                                      ci(*[m[2] for m in members]), cd(*[m[3] for m in members]),
                                      cd(*[m[4] for m in members]), dzp, ci(*[BC[m[6]] for m in members]),
                                      int(nstreams), int(bool(autotune)), stream)
        _check(st, "flups_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().flups_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, fs, ps, rtol=1e-10, max_iter=4, info=True, check=True):
        n = self.n
        fa = (ctypes.c_void_p * n)(*[ptr(x) for x in fs])
        pa = (ctypes.c_void_p * n)(*[ptr(x) for x in ps])
        inf = (Info * n)() if info else None
        st = lib().flups_batch_solve(self._h, fa, pa, float(rtol), int(max_iter), inf)
        if check:
            _check(st, "flups_batch_solve")
            return list(inf) if inf is not None else None
        return st, (list(inf) if inf is not None else None)

    @property
    def graph_kernels(self):
        return lib().flups_batch_graph_kernels(self._h)

    def tuning(self, m):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().flups_batch_member_tuning(self._h, int(m), ctypes.byref(a), ctypes.byref(b)),
               "flups_batch_member_tuning")
        return a.value, b.value


def _fparams(params):
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
    if a.size != PNET_NPARAMS:
        raise ValueError(f"expected {PNET_NPARAMS} parameters, got {a.size}")
    return a


class PNet:
    """Learned splitting-pressure net on one periodic grid (flups_pnet_*).

    params: FLUPS_PNET_NPARAMS floats, per layer W[out][in][27] then b[out]."""

    def __init__(self, nx, ny, nz, params, stream=None):
        self.shape = (nz, ny, nx)
        if stream is None:
            stream = current_stream()
        a = _fparams(params)
        h = ctypes.c_void_p()
        st = lib().flups_pnet_create(ctypes.byref(h), int(nx), int(ny), int(nz),
                                     a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), stream)
        _check(st, "flups_pnet_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().flups_pnet_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def launches(self):
        return lib().flups_pnet_launch_count(self._h)

    def set_profiling(self, on=True):
        _check(lib().flups_pnet_set_profiling(self._h, int(bool(on))), "flups_pnet_set_profiling")

    def profile(self):
        """{kernel group: (total ms, timed regions)} since the last call (synchronises)."""
        ms = (ctypes.c_double * PNET_NKERNELS)()
        n = (ctypes.c_longlong * PNET_NKERNELS)()
        _check(lib().flups_pnet_profile_read(self._h, ms, n), "flups_pnet_profile_read")
        return {lib().flups_pnet_kernel_name(k).decode(): (ms[k], n[k]) for k in range(PNET_NKERNELS) if n[k]}

    def set_params(self, params):
        a = _fparams(params)
        _check(lib().flups_pnet_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "flups_pnet_set_params")

    def params(self):
        a = np.empty(PNET_NPARAMS, np.float32)
        _check(lib().flups_pnet_get_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "flups_pnet_get_params")
        return a

    def grads(self):
        a = np.empty(PNET_NPARAMS, np.float32)
        _check(lib().flups_pnet_get_grads(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "flups_pnet_get_grads")
        return a

    def adam_state(self):
        """(m, v, step): the Adam moments and the number of steps taken."""
        m = np.empty(PNET_NPARAMS, np.float32)
        v = np.empty(PNET_NPARAMS, np.float32)
        step = ctypes.c_longlong()
        fp = ctypes.POINTER(ctypes.c_float)
        _check(lib().flups_pnet_get_adam(self._h, m.ctypes.data_as(fp), v.ctypes.data_as(fp), ctypes.byref(step)),
               "flups_pnet_get_adam")
        return m, v, int(step.value)

    def set_adam_state(self, m, v, step):
        """Restore the Adam moments and step count (after set_params, which resets them)."""
        m, v = _fparams(m), _fparams(v)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(lib().flups_pnet_set_adam(self._h, m.ctypes.data_as(fp), v.ctypes.data_as(fp), int(step)),
               "flups_pnet_set_adam")

    def predict(self, rho, rho0, pn, pnm1, p_hat):
        _check(lib().flups_pnet_predict(self._h, ptr(rho), float(rho0), ptr(pn), ptr(pnm1), ptr(p_hat)),
               "flups_pnet_predict")

    def train_step(self, rho, rho0, pn, pnm1, pnext, lr, want_loss=True):
        loss = ctypes.c_double()
        _check(lib().flups_pnet_train_step(self._h, ptr(rho), float(rho0), ptr(pn), ptr(pnm1), ptr(pnext),
                                           float(lr), ctypes.byref(loss) if want_loss else None),
               "flups_pnet_train_step")
        return loss.value if want_loss else None

    def eval_loss(self, rho, rho0, pn, pnm1, pnext):
        loss = ctypes.c_double()
        _check(lib().flups_pnet_eval_loss(self._h, ptr(rho), float(rho0), ptr(pn), ptr(pnm1), ptr(pnext),
                                          ctypes.byref(loss)), "flups_pnet_eval_loss")
        return loss.value
