"""Python binding of the ztoep C-ABI (libztoep.so): argument marshalling only.

The functions carry the C names (`ztoep_plan`, `ztoep_matvec`, `ztoep_solve`,
...) and take torch tensors (device complex128, or host complex128 for
`ztoep_solve_host`) plus an optional torch CUDA stream.  Every step of the
computation runs in the library's CUDA kernels; there is no CPU fallback:
if the library is missing or fails to load, `lib()` raises.

`Plan` is a small owner object around a plan handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libztoep.so")

ZTOEP_OK = 0
ZTOEP_ERR_ARG = 1
ZTOEP_ERR_NOMEM = 2
ZTOEP_ERR_CUDA = 3
ZTOEP_ERR_NOCONV = 4
ZTOEP_ERR_TIMEOUT = 5
ZTOEP_ERR_UNSUPPORTED = 6
ZTOEP_ERR_NONFINITE = 7
ZTOEP_FP64 = 0
ZTOEP_MIXED = 1
ZTOEP_FLAG_ZERO_GUESS = 1
ZTOEP_FLAG_HOST_LOOP = 2


class ZtoepError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {ztoep_status_string(status)} ({status})")


class Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("b", ctypes.c_int32),
                ("n_edge", ctypes.c_int32), ("active", ctypes.c_void_p),
                ("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("edge_per_cell", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("prec", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("timeout_ns", ctypes.c_int64), ("flags", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("inner_iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("second_passes", ctypes.c_int32), ("rel_residual", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("b", ctypes.c_int32),
                ("n_edge", ctypes.c_int32), ("lx", ctypes.c_int32), ("ly", ctypes.c_int32),
                ("n_toep", ctypes.c_int64), ("n", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("resident_bytes", ctypes.c_size_t), ("dense_bytes", ctypes.c_size_t)]


class TuneInfo(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("rad_order_x", ctypes.c_int32),
                ("rad_order_y", ctypes.c_int32), ("fft_channels_x", ctypes.c_int32), ("fft_threads_x", ctypes.c_int32),
                ("fft_channels_y", ctypes.c_int32), ("fft_threads_y", ctypes.c_int32), ("fft_kernel_x", ctypes.c_int32),
                ("fft_kernel_y", ctypes.c_int32), ("bp_split", ctypes.c_int32),
                ("bp_ctas_per_sm", ctypes.c_int32), ("tc_kchunk", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("product_us", ctypes.c_double), ("default_us", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SchedOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("workers", ctypes.c_int32), ("device", ctypes.c_int32),
                ("fake_backend", ctypes.c_int32), ("fake_us", ctypes.c_int64), ("group_max", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("desc", Desc), ("inputs_on_device", ctypes.c_int32), ("plan_key", ctypes.c_uint64),
                ("T", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p), ("nrhs", ctypes.c_int32),
                ("V", ctypes.c_void_p), ("X", ctypes.c_void_p), ("opts", SolveOpts),
                ("info", ctypes.POINTER(SolveInfo))]


class RequestState(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("plan_reused", ctypes.c_int32),
                ("inputs_consumed", ctypes.c_int32), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class SchedStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("max_in_flight", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("resident_plan_bytes", ctypes.c_size_t), ("plans_built", ctypes.c_int64),
                ("plans_reused", ctypes.c_int64), ("plans_evicted", ctypes.c_int64), ("groups", ctypes.c_int64)]


_lib = None
c_p = ctypes.c_void_p
c_i32 = ctypes.c_int32

EXPORTS = ["ztoep_default_opts", "ztoep_plan", "ztoep_matvec", "ztoep_solve", "ztoep_solve_host",
           "ztoep_forward_spectrum", "ztoep_plan_spectrum", "ztoep_plan_get_info", "ztoep_footprint",
           "ztoep_plan_destroy", "ztoep_status_string", "ztoep_version", "ztoep_launch_count",
           "ztoep_timing_enable", "ztoep_timing_reset", "ztoep_timing_read", "ztoep_edge_product_noalloc",
           "ztoep_port_matrices", "ztoep_far_field_grid", "ztoep_solve_schur",
           "ztoep_sched_create", "ztoep_sched_submit", "ztoep_sched_poll", "ztoep_sched_wait",
           "ztoep_sched_get_stats", "ztoep_sched_destroy", "ztoep_plan_autotune", "ztoep_plan_tuned",
           "ztoep_plan_get_tune", "ztoep_solve_group"]

K_FFT, K_BLOCKPROD, K_EDGE, K_ARNOLDI, K_MISC, K_TENSOR, K_TENSOR_PIPE = range(7)
ZTOEP_TIMING_SERIAL = 1 << 30  # products run their branches one after another while timed


def lib(path: str | None = None):
    """Load libztoep.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libztoep.so not built ({p}); run __graft_entry__.build()")
    L = ctypes.CDLL(p)
    L.ztoep_default_opts.argtypes = [ctypes.POINTER(SolveOpts)]
    L.ztoep_default_opts.restype = c_i32
    L.ztoep_plan.argtypes = [ctypes.POINTER(Desc), c_p, c_p, c_p, c_p, ctypes.POINTER(c_p)]
    L.ztoep_plan.restype = c_i32
    L.ztoep_matvec.argtypes = [c_p, c_i32, c_i32, c_p, c_p, c_p]
    L.ztoep_matvec.restype = c_i32
    L.ztoep_solve.argtypes = [c_p, ctypes.POINTER(SolveOpts), c_i32, c_p, c_p, ctypes.POINTER(SolveInfo), c_p]
    L.ztoep_solve.restype = c_i32
    L.ztoep_solve_host.argtypes = [c_p, ctypes.POINTER(SolveOpts), c_i32, c_p, c_p, ctypes.POINTER(SolveInfo),
                                   c_p]
    L.ztoep_solve_host.restype = c_i32
    L.ztoep_solve_group.argtypes = [c_i32, ctypes.POINTER(c_p), ctypes.POINTER(SolveOpts), ctypes.POINTER(c_i32),
                                    ctypes.POINTER(c_p), ctypes.POINTER(c_p),
                                    ctypes.POINTER(ctypes.POINTER(SolveInfo)), c_p]
    L.ztoep_solve_group.restype = c_i32
    L.ztoep_forward_spectrum.argtypes = [c_p, c_i32, c_i32, c_p, c_p, c_p]
    L.ztoep_forward_spectrum.restype = c_i32
    L.ztoep_plan_spectrum.argtypes = [c_p, c_p, c_p]
    L.ztoep_plan_spectrum.restype = c_i32
    L.ztoep_plan_get_info.argtypes = [c_p, ctypes.POINTER(PlanInfo)]
    L.ztoep_plan_get_info.restype = c_i32
    L.ztoep_solve_schur.argtypes = [c_p, c_i32, c_p, c_p, ctypes.POINTER(SolveOpts), c_i32, c_p, c_p,
                                    ctypes.POINTER(SolveInfo), c_p]
    L.ztoep_solve_schur.restype = c_i32
    L.ztoep_far_field_grid.argtypes = [c_p, c_i32, c_p, c_i32, c_p, ctypes.c_double, ctypes.c_double, c_p, c_p]
    L.ztoep_far_field_grid.restype = c_i32
    L.ztoep_port_matrices.argtypes = [c_i32, ctypes.c_int64, c_p, c_p, c_p, c_p, c_p, c_p, c_p]
    L.ztoep_port_matrices.restype = c_i32
    L.ztoep_footprint.argtypes = [ctypes.POINTER(Desc), c_i32, c_i32]
    L.ztoep_footprint.restype = ctypes.c_size_t
    L.ztoep_plan_destroy.argtypes = [c_p]
    L.ztoep_plan_destroy.restype = None
    L.ztoep_status_string.argtypes = [c_i32]
    L.ztoep_status_string.restype = ctypes.c_char_p
    L.ztoep_version.argtypes = []
    L.ztoep_version.restype = ctypes.c_char_p
    L.ztoep_sched_create.argtypes = [ctypes.POINTER(SchedOpts), ctypes.POINTER(c_p)]
    L.ztoep_sched_create.restype = c_i32
    L.ztoep_sched_submit.argtypes = [c_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]
    L.ztoep_sched_submit.restype = c_i32
    L.ztoep_sched_poll.argtypes = [c_p, ctypes.c_int64, ctypes.POINTER(RequestState)]
    L.ztoep_sched_poll.restype = c_i32
    L.ztoep_sched_wait.argtypes = [c_p, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(RequestState)]
    L.ztoep_sched_wait.restype = c_i32
    L.ztoep_sched_get_stats.argtypes = [c_p, ctypes.POINTER(SchedStats)]
    L.ztoep_sched_get_stats.restype = c_i32
    L.ztoep_sched_destroy.argtypes = [c_p]
    L.ztoep_sched_destroy.restype = None
    L.ztoep_plan_autotune.argtypes = [ctypes.POINTER(Desc), c_p, c_p, c_p, c_i32, c_p, ctypes.POINTER(c_p),
                                      ctypes.POINTER(TuneInfo)]
    L.ztoep_plan_autotune.restype = c_i32
    L.ztoep_plan_tuned.argtypes = [ctypes.POINTER(Desc), c_p, c_p, c_p, ctypes.POINTER(TuneInfo), c_p,
                                   ctypes.POINTER(c_p)]
    L.ztoep_plan_tuned.restype = c_i32
    L.ztoep_plan_get_tune.argtypes = [c_p, ctypes.POINTER(TuneInfo)]
    L.ztoep_plan_get_tune.restype = c_i32
    L.ztoep_edge_product_noalloc.argtypes = [c_p, c_i32, c_p, c_p, c_p]
    L.ztoep_edge_product_noalloc.restype = c_i32
    L.ztoep_launch_count.argtypes = []
    L.ztoep_launch_count.restype = ctypes.c_uint64
    L.ztoep_timing_enable.argtypes = [c_i32]
    L.ztoep_timing_enable.restype = None
    L.ztoep_timing_reset.argtypes = []
    L.ztoep_timing_reset.restype = None
    L.ztoep_timing_read.argtypes = [c_i32, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]
    L.ztoep_timing_read.restype = c_i32
    if path is None:
        _lib = L
    return L


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    if t is None:
        return None
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous(), \
        "expected a contiguous CUDA complex128 tensor"
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    import torch
    if isinstance(a, torch.Tensor):
        assert (not a.is_cuda) and a.dtype == torch.complex128 and a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def make_desc(nx, ny, b, n_edge, active=None, lx=0, ly=0, edge_per_cell=0):
    """Returns (Desc, keepalive) -- keep the second item alive while the Desc is used."""
    keep = None
    ap = None
    if active is not None:
        keep = np.ascontiguousarray(np.asarray(active, dtype=np.uint8).reshape(-1))
        assert keep.size == nx * ny
        ap = keep.ctypes.data
    return Desc(nx, ny, b, n_edge, ap, lx, ly, edge_per_cell), keep


def _check(st, what):
    if st != ZTOEP_OK:
        raise ZtoepError(st, what)


def ztoep_version() -> str:
    return lib().ztoep_version().decode()


def ztoep_status_string(status: int) -> str:
    return lib().ztoep_status_string(status).decode()


def ztoep_default_opts() -> SolveOpts:
    o = SolveOpts()
    _check(lib().ztoep_default_opts(ctypes.byref(o)), "ztoep_default_opts")
    return o


def ztoep_plan(desc: Desc, T, B, C, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().ztoep_plan(ctypes.byref(desc), _dptr(T), _dptr(B), _dptr(C), _stream_ptr(stream),
                            ctypes.byref(h)), "ztoep_plan")
    return h


def ztoep_plan_autotune(desc: Desc, T, B, C, nrhs: int, stream=None) -> tuple[ctypes.c_void_p, TuneInfo]:
    h = ctypes.c_void_p()
    t = TuneInfo()
    _check(lib().ztoep_plan_autotune(ctypes.byref(desc), _dptr(T), _dptr(B), _dptr(C), nrhs, _stream_ptr(stream),
                                     ctypes.byref(h), ctypes.byref(t)), "ztoep_plan_autotune")
    return h, t


def ztoep_plan_tuned(desc: Desc, T, B, C, tune: TuneInfo, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().ztoep_plan_tuned(ctypes.byref(desc), _dptr(T), _dptr(B), _dptr(C), ctypes.byref(tune),
                                  _stream_ptr(stream), ctypes.byref(h)), "ztoep_plan_tuned")
    return h


def ztoep_plan_get_tune(plan) -> TuneInfo:
    t = TuneInfo()
    _check(lib().ztoep_plan_get_tune(plan, ctypes.byref(t)), "ztoep_plan_get_tune")
    return t


def ztoep_matvec(plan, prec: int, nrhs: int, X, Y, stream=None) -> int:
    return lib().ztoep_matvec(plan, prec, nrhs, _dptr(X), _dptr(Y), _stream_ptr(stream))


def ztoep_solve(plan, opts: SolveOpts, nrhs: int, V, X, info=None, stream=None) -> int:
    ip = info if info is not None else None
    return lib().ztoep_solve(plan, ctypes.byref(opts), nrhs, _dptr(V), _dptr(X), ip, _stream_ptr(stream))


def ztoep_solve_host(plan, opts: SolveOpts, nrhs: int, V_host, X_host, info=None, stream=None) -> int:
    ip = info if info is not None else None
    return lib().ztoep_solve_host(plan, ctypes.byref(opts), nrhs, _hptr(V_host), _hptr(X_host), ip,
                                  _stream_ptr(stream))


def ztoep_solve_group(plans, opts: SolveOpts, V, X, infos=None, stream=None) -> int:
    """One solve of several systems (plans of any sizes): V[i], X[i] device
    complex128 [nrhs_i][N_i]; infos[i] an info_array(nrhs_i) or None."""
    n = len(plans)
    P = (c_p * n)(*[p.value if isinstance(p, c_p) else p for p in plans])
    R = (c_i32 * n)(*[int(v.shape[0]) for v in V])
    VP = (c_p * n)(*[_dptr(v) for v in V])
    XP = (c_p * n)(*[_dptr(x) for x in X])
    IP = None
    if infos is not None:
        IP = (ctypes.POINTER(SolveInfo) * n)(*[ctypes.cast(i, ctypes.POINTER(SolveInfo)) if i is not None
                                               else ctypes.POINTER(SolveInfo)() for i in infos])
    return lib().ztoep_solve_group(n, P, ctypes.byref(opts), R, VP, XP, IP, _stream_ptr(stream))


def ztoep_forward_spectrum(plan, prec: int, nrhs: int, X, Xhat, stream=None) -> int:
    return lib().ztoep_forward_spectrum(plan, prec, nrhs, _dptr(X), _dptr(Xhat), _stream_ptr(stream))


def ztoep_plan_spectrum(plan, That, stream=None) -> int:
    return lib().ztoep_plan_spectrum(plan, _dptr(That), _stream_ptr(stream))


def ztoep_plan_get_info(plan) -> PlanInfo:
    info = PlanInfo()
    _check(lib().ztoep_plan_get_info(plan, ctypes.byref(info)), "ztoep_plan_get_info")
    return info


def ztoep_port_matrices(p: int, n: int, I, ports, edge_len, z0, Y, S, stream=None) -> int:
    """Argument marshalling for ztoep_port_matrices: I, Y, S device complex128
    tensors; ports (int32), edge_len and z0 (float64) host numpy arrays."""
    import numpy as np
    pa = np.ascontiguousarray(ports, dtype=np.int32)
    la = np.ascontiguousarray(edge_len, dtype=np.float64)
    za = np.ascontiguousarray(z0, dtype=np.float64)
    return lib().ztoep_port_matrices(p, n, _dptr(I), pa.ctypes.data_as(c_p), la.ctypes.data_as(c_p),
                                     za.ctypes.data_as(c_p), _dptr(Y), _dptr(S), _stream_ptr(stream))


def ztoep_solve_schur(plan_A, n_edge: int, B, C, opts: SolveOpts, nrhs: int, V, X, info=None, stream=None) -> int:
    return lib().ztoep_solve_schur(plan_A, n_edge, _dptr(B), _dptr(C), ctypes.byref(opts), nrhs, _dptr(V), _dptr(X),
                                   info, _stream_ptr(stream))


def ztoep_far_field_grid(plan, nrhs: int, I, npol: int, Fh, k: float, eta: float, F, stream=None) -> int:
    return lib().ztoep_far_field_grid(plan, nrhs, _dptr(I), npol, _dptr(Fh), k, eta, _dptr(F), _stream_ptr(stream))


def port_matrices(I, ports, edge_len, z0, stream=None):
    """(Y, S) for the delta-port solutions I ([p][n] complex128 on the
    device, row k solved for port k); raises ZtoepError on a bad status."""
    import torch
    p, n = I.shape
    Y = torch.empty((p, p), dtype=torch.complex128, device=I.device)
    S = torch.empty_like(Y)
    st = ztoep_port_matrices(p, n, I, ports, edge_len, z0, Y, S, stream)
    if st != 0:
        raise ZtoepError(st)
    return Y, S


def ztoep_footprint(desc: Desc, max_nrhs: int, restart: int = 30) -> int:
    return lib().ztoep_footprint(ctypes.byref(desc), max_nrhs, restart)


def ztoep_plan_destroy(plan) -> None:
    lib().ztoep_plan_destroy(plan)


def ztoep_edge_product_noalloc(plan, nrhs: int, X, Y, stream=None) -> int:
    """Edge-coupling part of the FP64 product with no device allocation (for
    callers that cannot allocate at call time, e.g. hosts that forbid allocation
    after start-up); scratch is a fixed 16 MiB device array shared by all calls."""
    return lib().ztoep_edge_product_noalloc(plan, nrhs, _dptr(X), _dptr(Y), _stream_ptr(stream))


def ztoep_launch_count() -> int:
    return int(lib().ztoep_launch_count())


def ztoep_timing_enable(mask: int) -> None:
    lib().ztoep_timing_enable(mask)


def ztoep_timing_reset() -> None:
    lib().ztoep_timing_reset()


def ztoep_timing_read(cls: int) -> tuple[int, float]:
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(lib().ztoep_timing_read(cls, ctypes.byref(n), ctypes.byref(ms)), "ztoep_timing_read")
    return int(n.value), float(ms.value)


def ztoep_sched_create(opts: SchedOpts):
    h = ctypes.c_void_p()
    _check(lib().ztoep_sched_create(ctypes.byref(opts), ctypes.byref(h)), "ztoep_sched_create")
    return h


def ztoep_sched_submit(sched, req: Request) -> tuple[int, int]:
    rid = ctypes.c_int64(-1)
    st = lib().ztoep_sched_submit(sched, ctypes.byref(req), ctypes.byref(rid))
    return st, int(rid.value)


def ztoep_sched_poll(sched, rid: int) -> RequestState:
    st = RequestState()
    _check(lib().ztoep_sched_poll(sched, rid, ctypes.byref(st)), "ztoep_sched_poll")
    return st


def ztoep_sched_wait(sched, rid: int, timeout_ms: int = -1) -> tuple[int, RequestState]:
    st = RequestState()
    rc = lib().ztoep_sched_wait(sched, rid, timeout_ms, ctypes.byref(st))
    return rc, st


def ztoep_sched_get_stats(sched) -> SchedStats:
    st = SchedStats()
    _check(lib().ztoep_sched_get_stats(sched, ctypes.byref(st)), "ztoep_sched_get_stats")
    return st


def ztoep_sched_destroy(sched) -> None:
    lib().ztoep_sched_destroy(sched)


class Scheduler:
    """Owner of a serving scheduler; keeps every submitted request's buffers
    alive until the request is done."""

    def __init__(self, hbm_budget: int, workers: int = 4, device: int = 0, fake_us: int | None = None,
                 group_max: int = 1):
        o = SchedOpts(hbm_budget, workers, device, 1 if fake_us is not None else 0, fake_us or 0, group_max)
        self.handle = ztoep_sched_create(o)
        self._keep = {}

    def submit(self, desc_args, T, B, C, V, X, opts: SolveOpts | None = None, plan_key: int = 0,
               on_device: bool | None = None):
        """desc_args = (nx, ny, b, n_edge, active, lx, ly); arrays are torch tensors
        (all on the device or all on the host) or numpy arrays (host)."""
        import torch
        desc, keep = make_desc(*desc_args)
        if on_device is None:
            on_device = isinstance(V, torch.Tensor) and V.is_cuda

        def ptr(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return ctypes.c_void_p(a.data_ptr())
            return ctypes.c_void_p(a.ctypes.data)

        nrhs = V.shape[0]
        info = info_array(nrhs)
        req = Request(desc, 1 if on_device else 0, plan_key, ptr(T), ptr(B), ptr(C), nrhs, ptr(V), ptr(X),
                      opts or ztoep_default_opts(), info)
        st, rid = ztoep_sched_submit(self.handle, req)
        if st != ZTOEP_OK:
            raise ZtoepError(st, "ztoep_sched_submit")
        self._keep[rid] = (keep, T, B, C, V, X, info, req)
        return rid

    def wait(self, rid: int, timeout_ms: int = -1):
        rc, st = ztoep_sched_wait(self.handle, rid, timeout_ms)
        info = self._keep[rid][6]
        return rc, st, [dict(outer=i.outer, inner_iters=i.inner_iters, status=i.status,
                             rel_residual=i.rel_residual) for i in info]

    def poll(self, rid: int) -> RequestState:
        return ztoep_sched_poll(self.handle, rid)

    def drop_inputs(self, rid: int) -> bool:
        """Forget the request's T, B, C once the scheduler reports them consumed;
        returns whether it did."""
        k = self._keep.get(rid)
        if k is None or k[1] is None:
            return True
        if not ztoep_sched_poll(self.handle, rid).inputs_consumed:
            return False
        self._keep[rid] = (k[0], None, None, None) + k[4:]
        return True

    def release(self, rid: int):
        self._keep.pop(rid, None)

    def stats(self) -> SchedStats:
        return ztoep_sched_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            ztoep_sched_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def info_array(nrhs: int):
    return (SolveInfo * nrhs)()


class Plan:
    """Owns a plan built from a synthetic Problem (or explicit arrays)."""

    def __init__(self, nx, ny, b, n_edge, T, B, C, active=None, lx=0, ly=0, stream=None, autotune: int = 0,
                 tune: TuneInfo | None = None, edge_per_cell: int = 0):
        """autotune > 0: ztoep_plan_autotune for that many RHS; tune: ztoep_plan_tuned;
        edge_per_cell > 0: B has the perimeter side-Toeplitz layout (see ztoep.h)."""
        self.desc, self._keep = make_desc(nx, ny, b, n_edge, active, lx, ly, edge_per_cell)
        self.tune = None
        if autotune:
            self.handle, self.tune = ztoep_plan_autotune(self.desc, T, B, C, autotune, stream)
        elif tune is not None:
            self.handle = ztoep_plan_tuned(self.desc, T, B, C, tune, stream)
        else:
            self.handle = ztoep_plan(self.desc, T, B, C, stream)
        self.info = ztoep_plan_get_info(self.handle)
        self.n = int(self.info.n)

    @classmethod
    def from_problem(cls, prob, device="cuda", lx=0, ly=0, stream=None, autotune: int = 0, tune=None,
                     structured: bool = False):
        """structured: declare the problem's perimeter edge layout (prob.edge_per_cell) to the plan."""
        import torch
        T = torch.from_numpy(np.ascontiguousarray(prob.T)).to(device)
        B = torch.from_numpy(np.ascontiguousarray(prob.B)).to(device) if prob.n_edge else None
        C = torch.from_numpy(np.ascontiguousarray(prob.C)).to(device) if prob.n_edge else None
        act = prob.active if not prob.active.all() else None
        k = prob.edge_per_cell if structured else 0
        if structured and not k:
            raise ValueError("the problem's edge layout is not the perimeter side-Toeplitz one")
        p = cls(prob.nx, prob.ny, prob.b, prob.n_edge, T, B, C, act, lx, ly, stream, autotune, tune, k)
        if stream is None:
            torch.cuda.current_stream().synchronize()
        else:
            stream.synchronize()
        return p

    def matvec(self, X, prec=ZTOEP_FP64, stream=None):
        import torch
        Y = torch.empty_like(X)
        _check(ztoep_matvec(self.handle, prec, X.shape[0], X, Y, stream), "ztoep_matvec")
        return Y

    def solve(self, V, X=None, opts: SolveOpts | None = None, stream=None, check=True):
        import torch
        o = opts or ztoep_default_opts()
        nrhs = V.shape[0]
        if X is None:
            X = torch.zeros_like(V)
            o.flags |= ZTOEP_FLAG_ZERO_GUESS
        info = info_array(nrhs)
        st = ztoep_solve(self.handle, o, nrhs, V, X, info, stream)
        if check and st not in (ZTOEP_OK,):
            raise ZtoepError(st, "ztoep_solve")
        return X, [dict(outer=i.outer, inner_iters=i.inner_iters, status=i.status,
                        second_passes=i.second_passes, rel_residual=i.rel_residual) for i in info], st

    def far_field(self, I, Fh, k: float, eta: float, stream=None):
        """Far field on the array-factor grid (ztoep_far_field_grid): I
        [nrhs][N], Fh [lx*ly][npol][b] device complex128 -> [nrhs][lx*ly][npol]."""
        import torch
        nrhs, npol = I.shape[0], Fh.shape[1]
        F = torch.empty((nrhs, Fh.shape[0], npol), dtype=torch.complex128, device=I.device)
        st = ztoep_far_field_grid(self.handle, nrhs, I, npol, Fh, k, eta, F, stream)
        if st != 0:
            raise ZtoepError(st, "ztoep_far_field_grid")
        return F

    def close(self):
        if getattr(self, "handle", None):
            ztoep_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
