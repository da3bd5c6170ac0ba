"""Thin ctypes binding of the C ABI in ``include/hse.h``.

Every function here only marshals arguments to the CUDA library
``libhse.so``; all of the computation runs in its kernels on the GPU.  The
functions carry the C names.  ``Plan`` is a small convenience wrapper that
takes torch CUDA tensors (component-major float64) and passes their device
pointers and the current stream.  If the library cannot be loaded, importing
the entry points raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HSE_OK, HSE_ERR_INVALID, HSE_ERR_OOM, HSE_ERR_CUDA, HSE_ERR_CUFFT, HSE_ERR_TIMEOUT, HSE_ERR_UNSUPPORTED = range(7)
HSE_STOKESLET, HSE_STRESSLET, HSE_ROTLET, HSE_FREE_SPACE = 1, 2, 4, 8
HSE_FP64, HSE_MIXED = 0, 1
HSE_FFT_AUTO, HSE_FFT_CUFFT, HSE_FFT_DF64 = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhse.so")


class hse_params(ctypes.Structure):
    _fields_ = [
        ("kernel_mask", ctypes.c_int), ("precision", ctypes.c_int), ("box", ctypes.c_double * 3),
        ("L", ctypes.c_double), ("xi", ctypes.c_double), ("rc", ctypes.c_double), ("rc64", ctypes.c_double),
        ("P", ctypes.c_int),
        ("M", ctypes.c_int), ("Mt", ctypes.c_int), ("h", ctypes.c_double), ("eta", ctypes.c_double),
        ("ncell", ctypes.c_int * 3), ("n_fft_in", ctypes.c_int), ("n_fft_out", ctypes.c_int),
        ("fft", ctypes.c_int), ("grid_bytes", ctypes.c_size_t), ("spread_tile", ctypes.c_int * 3),
        ("rcmid", ctypes.c_double),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


HSE_N_STAGES = 8
STAGE_NAMES = ("check", "cells", "real", "spread", "fft", "scale", "ifft", "gather")


class hse_eval_stats(ctypes.Structure):
    _fields_ = [("n_kernel_launches", ctypes.c_int), ("n_fft_execs", ctypes.c_int), ("timing", ctypes.c_int),
                ("stage_ms", ctypes.c_double * HSE_N_STAGES), ("overlapped", ctypes.c_int),
                ("total_ms", ctypes.c_double)]


HSE_PENDING = 7


class hse_server_config(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t)]


class hse_request(ctypes.Structure):
    _fields_ = [("kernel_mask", ctypes.c_int), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("box", ctypes.c_double * 3), ("n_src", ctypes.c_int64), ("src_xyz", ctypes.c_void_p),
                ("strengths", ctypes.c_void_p), ("n_tgt", ctypes.c_int64), ("tgt_xyz", ctypes.c_void_p),
                ("vel", ctypes.c_void_p)]


class hse_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("busy_s", ctypes.c_double), ("targets_per_s", ctypes.c_double),
                ("plans_created", ctypes.c_int64), ("plans_evicted", ctypes.c_int64),
                ("resident_bytes", ctypes.c_size_t), ("plan_hits", ctypes.c_int64), ("plan_build_s", ctypes.c_double)]


class hse_instance(ctypes.Structure):
    _fields_ = [("kernel_mask", ctypes.c_int), ("n", ctypes.c_int64), ("src_xyz", ctypes.c_void_p),
                ("strengths", ctypes.c_void_p), ("vel", ctypes.c_void_p)]


class hse_batch_stats(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int64), ("particles", ctypes.c_int64), ("chunks", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("fft_execs", ctypes.c_int64), ("plans", ctypes.c_int64),
                ("autotuned_groups", ctypes.c_int64), ("grid_bytes", ctypes.c_size_t),
                ("fft_work_bytes", ctypes.c_size_t), ("particle_bytes", ctypes.c_size_t),
                ("plan_bytes", ctypes.c_size_t), ("stage_ms", ctypes.c_double * 8),
                ("graphs_captured", ctypes.c_int64), ("graph_launches", ctypes.c_int64)]


class hse_pipe_peaks(ctypes.Structure):
    _fields_ = [("fp64_tflops", ctypes.c_double), ("fp32_tflops", ctypes.c_double), ("df64_tflops", ctypes.c_double),
                ("n_sm", ctypes.c_int), ("sm_clock_mhz", ctypes.c_double)]


class HseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_lib = None
_NAMES = ("hse_plan_create", "hse_plan_set_grid", "hse_plan_set_rc64", "hse_plan_set_rcmid", "hse_plan_set_fft", "hse_plan_get_params", "hse_eval", "hse_eval_parts",
          "hse_cell_list", "hse_neighbor_counts", "hse_spread_grids", "hse_plan_destroy", "hse_status_string",
          "hse_last_error", "hse_plan_set_timing", "hse_plan_set_overlap", "hse_plan_set_real_residency", "hse_plan_set_spread_tile", "hse_get_eval_stats", "hse_cell_list_noalloc",
          "hse_server_create", "hse_server_submit", "hse_server_poll", "hse_server_wait", "hse_server_get_stats",
          "hse_server_reset_stats", "hse_server_destroy", "hse_server_error_text", "hse_server_prewarm",
          "hse_server_request_params", "hse_batch_create",
          "hse_batch_eval", "hse_batch_get_stats", "hse_batch_instance_params", "hse_batch_last_error", "hse_batch_destroy",
          "hse_batch_set_timing", "hse_batch_set_graphs", "hse_measure_pipe_peaks")


def load(path: str = LIB_PATH):
    """Load libhse.so (raises OSError when it is absent: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"CUDA library {path} is missing; build it with paper_1802_07844_gb300.build")
    L = ctypes.CDLL(path)
    vp, dp, i64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64
    L.hse_plan_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(vp)]
    L.hse_plan_set_grid.argtypes = [vp, ctypes.c_int]
    L.hse_plan_set_rc64.argtypes = [vp, ctypes.c_double]
    L.hse_plan_set_rcmid.argtypes = [vp, ctypes.c_double]
    L.hse_plan_set_fft.argtypes = [vp, ctypes.c_int]
    L.hse_plan_get_params.argtypes = [vp, ctypes.POINTER(hse_params)]
    L.hse_eval.argtypes = [vp, i64, dp, dp, i64, dp, dp, vp]
    L.hse_eval_parts.argtypes = [vp, i64, dp, dp, i64, dp, dp, dp, vp]
    L.hse_cell_list.argtypes = [vp, i64, dp, dp, dp, dp, vp]
    L.hse_neighbor_counts.argtypes = [vp, i64, dp, i64, dp, dp, dp, vp]
    L.hse_spread_grids.argtypes = [vp, i64, dp, dp, dp, ctypes.POINTER(ctypes.c_int), vp]
    L.hse_plan_destroy.argtypes = [vp]
    L.hse_plan_set_timing.argtypes = [vp, ctypes.c_int]
    L.hse_plan_set_overlap.argtypes = [vp, ctypes.c_int]
    L.hse_plan_set_real_residency.argtypes = [vp, ctypes.c_int]
    L.hse_plan_set_spread_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hse_server_create.argtypes = [ctypes.POINTER(hse_server_config), ctypes.POINTER(vp)]
    L.hse_server_submit.argtypes = [vp, ctypes.POINTER(hse_request), ctypes.POINTER(ctypes.c_uint64)]
    L.hse_server_poll.argtypes = [vp, ctypes.c_uint64]
    L.hse_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double]
    L.hse_server_get_stats.argtypes = [vp, ctypes.POINTER(hse_server_stats)]
    L.hse_server_reset_stats.argtypes = [vp]
    L.hse_server_destroy.argtypes = [vp]
    L.hse_server_prewarm.argtypes = [vp, ctypes.POINTER(hse_request)]
    L.hse_server_request_params.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(hse_params)]
    L.hse_server_error_text.argtypes = [vp, ctypes.c_uint64]
    L.hse_server_error_text.restype = ctypes.c_char_p
    L.hse_batch_create.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                                   ctypes.c_int, ctypes.POINTER(vp)]
    L.hse_batch_eval.argtypes = [vp, ctypes.c_int, ctypes.POINTER(hse_instance), vp]
    L.hse_batch_get_stats.argtypes = [vp, ctypes.POINTER(hse_batch_stats)]
    L.hse_batch_instance_params.argtypes = [vp, ctypes.c_int, ctypes.POINTER(hse_params)]
    L.hse_batch_last_error.argtypes = [vp]
    L.hse_batch_last_error.restype = ctypes.c_char_p
    L.hse_batch_destroy.argtypes = [vp]
    L.hse_batch_set_timing.argtypes = [vp, ctypes.c_int]
    L.hse_batch_set_graphs.argtypes = [vp, ctypes.c_int]
    L.hse_cell_list_noalloc.argtypes = [i64, dp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), dp, dp,
                                        dp, vp]
    L.hse_get_eval_stats.argtypes = [vp, ctypes.POINTER(hse_eval_stats)]
    L.hse_measure_pipe_peaks.argtypes = [ctypes.POINTER(hse_pipe_peaks)]
    L.hse_status_string.argtypes = [ctypes.c_int]
    L.hse_status_string.restype = ctypes.c_char_p
    L.hse_last_error.argtypes = [vp]
    L.hse_last_error.restype = ctypes.c_char_p
    for n in _NAMES:
        if getattr(L, n).restype is None and n not in ("hse_status_string", "hse_last_error", "hse_batch_last_error"):
            getattr(L, n).restype = ctypes.c_int
    _lib = L
    return L


def status_name(s: int) -> str:
    return load().hse_status_string(int(s)).decode()


def _check(status, plan=None):
    if status != HSE_OK:
        raise HseError(status, load().hse_last_error(plan).decode())


# ---------------------------------------------------------------- C names
def hse_plan_create(kernel_mask, box, xi, rc, P, tol, precision=HSE_FP64):
    L = load()
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    out = ctypes.c_void_p()
    _check(L.hse_plan_create(int(kernel_mask), b, float(xi), float(rc), int(P), float(tol), int(precision),
                             ctypes.byref(out)))
    return out


def hse_plan_set_rc64(plan, rc64):
    """FP64 plans: pairs closer than rc64 in FP64, the shell [rc64, rc) in FP32
    (rc64 >= rc: FP64 throughout)."""
    _check(load().hse_plan_set_rc64(plan, float(rc64)), plan)


def hse_plan_set_rcmid(plan, rcmid):
    _check(load().hse_plan_set_rcmid(plan, float(rcmid)), plan)


def hse_plan_set_fft(plan, mode):
    """Transforms of the Fourier part: HSE_FFT_AUTO, HSE_FFT_CUFFT or HSE_FFT_DF64."""
    _check(load().hse_plan_set_fft(plan, int(mode)), plan)


def hse_plan_set_grid(plan, M):
    _check(load().hse_plan_set_grid(plan, int(M)), plan)


def hse_plan_get_params(plan) -> dict:
    p = hse_params()
    _check(load().hse_plan_get_params(plan, ctypes.byref(p)), plan)
    return p.as_dict()


def hse_eval(plan, n_src, src_ptr, str_ptr, n_tgt, tgt_ptr, vel_ptr, stream=0):
    _check(load().hse_eval(plan, n_src, src_ptr, str_ptr, n_tgt, tgt_ptr, vel_ptr, stream), plan)


def hse_eval_parts(plan, n_src, src_ptr, str_ptr, n_tgt, tgt_ptr, real_ptr, four_ptr, stream=0):
    _check(load().hse_eval_parts(plan, n_src, src_ptr, str_ptr, n_tgt, tgt_ptr, real_ptr, four_ptr, stream), plan)


def hse_cell_list(plan, n, pos_ptr, cell_ptr, perm_ptr, start_ptr, stream=0):
    _check(load().hse_cell_list(plan, n, pos_ptr, cell_ptr, perm_ptr, start_ptr, stream), plan)


def hse_neighbor_counts(plan, n_src, src_ptr, n_tgt, tgt_ptr, a_ptr, b_ptr, stream=0):
    _check(load().hse_neighbor_counts(plan, n_src, src_ptr, n_tgt, tgt_ptr, a_ptr, b_ptr, stream), plan)


def hse_spread_grids(plan, n_src, src_ptr, str_ptr, grids_ptr, stream=0) -> int:
    n = ctypes.c_int()
    _check(load().hse_spread_grids(plan, n_src, src_ptr, str_ptr, grids_ptr, ctypes.byref(n), stream), plan)
    return n.value


def hse_plan_destroy(plan):
    _check(load().hse_plan_destroy(plan))


def hse_plan_set_timing(plan, enable):
    _check(load().hse_plan_set_timing(plan, int(bool(enable))), plan)


def hse_plan_set_overlap(plan, enable):
    _check(load().hse_plan_set_overlap(plan, int(bool(enable))), plan)


def hse_plan_set_real_residency(plan, blocks_per_sm):
    _check(load().hse_plan_set_real_residency(plan, int(blocks_per_sm)), plan)


def hse_plan_set_spread_tile(plan, wx, wy, wz):
    _check(load().hse_plan_set_spread_tile(plan, int(wx), int(wy), int(wz)), plan)


def hse_get_eval_stats(plan) -> dict:
    st = hse_eval_stats()
    _check(load().hse_get_eval_stats(plan, ctypes.byref(st)), plan)
    return {"n_kernel_launches": st.n_kernel_launches, "n_fft_execs": st.n_fft_execs, "timing": bool(st.timing),
            "stage_ms": dict(zip(STAGE_NAMES, list(st.stage_ms))), "overlapped": bool(st.overlapped),
            "total_ms": st.total_ms}


def hse_measure_pipe_peaks() -> dict:
    """Measured FP64, FP32 and df64 multiply-add throughput (TFLOP/s) of the current device."""
    p = hse_pipe_peaks()
    _check(load().hse_measure_pipe_peaks(ctypes.byref(p)))
    return {name: getattr(p, name) for name, _ in hse_pipe_peaks._fields_}


HSE_NOALLOC_MAX_POINTS = 262144


def hse_cell_list_noalloc(n, pos_ptr, box, ncell, cell_ptr, perm_ptr, start_ptr, stream=0):
    """Cell list without any device allocation (for callers whose allocator
    owns the device heap or that may not allocate in their loop)."""
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    c = (ctypes.c_int * 3)(*[int(v) for v in ncell])
    _check(load().hse_cell_list_noalloc(n, pos_ptr, b, c, cell_ptr, perm_ptr, start_ptr, stream))


def hse_server_create(n_slots, mem_budget_bytes=0):
    cfg = hse_server_config(int(n_slots), int(mem_budget_bytes))
    out = ctypes.c_void_p()
    _check(load().hse_server_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def hse_server_submit(srv, req: hse_request) -> int:
    t = ctypes.c_uint64()
    _check(load().hse_server_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def hse_server_poll(srv, ticket) -> int:
    return load().hse_server_poll(srv, ticket)


def hse_server_wait(srv, ticket, timeout_s) -> int:
    return load().hse_server_wait(srv, ticket, float(timeout_s))


def hse_server_get_stats(srv) -> dict:
    st = hse_server_stats()
    _check(load().hse_server_get_stats(srv, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in hse_server_stats._fields_}


def hse_server_reset_stats(srv):
    _check(load().hse_server_reset_stats(srv))


def hse_server_error_text(srv, ticket) -> str:
    return load().hse_server_error_text(srv, ticket).decode()


def hse_server_destroy(srv):
    _check(load().hse_server_destroy(srv))


def hse_server_prewarm(srv, req: hse_request):
    _check(load().hse_server_prewarm(srv, ctypes.byref(req)))


def hse_server_request_params(srv, ticket) -> dict:
    """Parameters of the plan that evaluated a finished request."""
    p = hse_params()
    st = load().hse_server_request_params(srv, ticket, ctypes.byref(p))
    if st != HSE_OK:
        raise HseError(st, f"request {ticket}: no parameters")
    return p.as_dict()


class Server:
    """Continuous-batching server; requests reference torch CUDA tensors that
    the caller keeps alive until completion."""

    def __init__(self, n_slots=3, mem_budget_bytes=0):
        self.handle = hse_server_create(n_slots, mem_budget_bytes)
        self._keep = {}

    def submit(self, kernel_mask, src, strengths, tol, precision=HSE_FP64, tgt=None, box=(1.0, 1.0, 1.0), out=None):
        import torch
        n_src = src.shape[1]
        n_tgt = n_src if tgt is None else tgt.shape[1]
        if out is None:
            out = torch.empty((3, n_tgt), dtype=torch.float64, device=src.device)
        req = hse_request(int(kernel_mask), int(precision), float(tol), (ctypes.c_double * 3)(*box), n_src,
                          Plan._ptr(src), Plan._ptr(strengths), n_tgt, Plan._ptr(tgt), Plan._ptr(out))
        t = hse_server_submit(self.handle, req)
        self._keep[t] = (src, strengths, tgt, out)
        return t

    def prewarm(self, kernel_mask, n_src, tol, precision=HSE_FP64, box=(1.0, 1.0, 1.0)):
        req = hse_request(int(kernel_mask), int(precision), float(tol), (ctypes.c_double * 3)(*box), int(n_src),
                          None, None, int(n_src), None, None)
        hse_server_prewarm(self.handle, req)

    def request_params(self, ticket):
        return hse_server_request_params(self.handle, ticket)

    def poll(self, ticket):
        return hse_server_poll(self.handle, ticket)

    def wait(self, ticket, timeout_s=600.0):
        st = hse_server_wait(self.handle, ticket, timeout_s)
        if st not in (HSE_OK, HSE_ERR_TIMEOUT):
            raise HseError(st, f"request {ticket} failed: {hse_server_error_text(self.handle, ticket)}")
        return st

    def result(self, ticket):
        return self._keep[ticket][3]

    def stats(self):
        return hse_server_get_stats(self.handle)

    def reset_stats(self):
        hse_server_reset_stats(self.handle)

    def close(self):
        if self.handle is not None:
            hse_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hse_batch_create(tol, precision=HSE_FP64, box=(1.0, 1.0, 1.0), mem_budget_bytes=0, autotune=0):
    out = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    _check(load().hse_batch_create(float(tol), int(precision), b, int(mem_budget_bytes), int(autotune),
                                   ctypes.byref(out)))
    return out


def hse_batch_last_error(batch) -> str:
    return load().hse_batch_last_error(batch).decode()


def hse_batch_eval(batch, instances, stream=0):
    """instances: a ctypes array of hse_instance (device pointers)."""
    st = load().hse_batch_eval(batch, len(instances), instances, stream)
    if st != HSE_OK:
        raise HseError(st, hse_batch_last_error(batch))


def hse_batch_get_stats(batch) -> dict:
    st = hse_batch_stats()
    _check(load().hse_batch_get_stats(batch, ctypes.byref(st)))
    out = {name: getattr(st, name) for name, _ in hse_batch_stats._fields_ if name != "stage_ms"}
    out["stage_ms"] = {STAGE_NAMES[i]: st.stage_ms[i] for i in range(8)}
    return out


def hse_batch_instance_params(batch, i) -> dict:
    p = hse_params()
    st = load().hse_batch_instance_params(batch, int(i), ctypes.byref(p))
    if st != HSE_OK:
        raise HseError(st, hse_batch_last_error(batch))
    return p.as_dict()


def hse_batch_set_timing(batch, enable):
    _check(load().hse_batch_set_timing(batch, 1 if enable else 0))


def hse_batch_set_graphs(batch, enable):
    _check(load().hse_batch_set_graphs(batch, 1 if enable else 0))


def hse_batch_destroy(batch):
    _check(load().hse_batch_destroy(batch))


class Batch:
    """Evaluates lists of independent instances (targets = sources) grouped by
    kernel mask and xi; every stage is one launch per chunk of instances."""

    def __init__(self, tol, precision=HSE_FP64, box=(1.0, 1.0, 1.0), mem_budget_bytes=0, autotune=False):
        self.handle = hse_batch_create(tol, precision, box, mem_budget_bytes, 1 if autotune else 0)

    def eval(self, items, outs=None):
        """items: list of (kernel_mask, src (3,n), strengths (rows,n)) torch CUDA
        float64 tensors.  Returns the list of (3,n) velocity tensors."""
        import torch
        arr = (hse_instance * len(items))()
        if outs is None:
            outs = [torch.empty((3, src.shape[1]), dtype=torch.float64, device=src.device) for _, src, _ in items]
        for i, (mask, src, strengths) in enumerate(items):
            arr[i] = hse_instance(int(mask), src.shape[1], Plan._ptr(src), Plan._ptr(strengths), Plan._ptr(outs[i]))
        stream = torch.cuda.current_stream().cuda_stream if items else 0
        hse_batch_eval(self.handle, arr, stream)
        return outs

    def stats(self):
        return hse_batch_get_stats(self.handle)

    def instance_params(self, i):
        return hse_batch_instance_params(self.handle, i)

    def set_timing(self, enable=True):
        hse_batch_set_timing(self.handle, enable)

    def set_graphs(self, enable=True):
        hse_batch_set_graphs(self.handle, enable)

    def close(self):
        if self.handle is not None:
            hse_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hse_status_string(status) -> str:
    return status_name(status)


def hse_last_error(plan=None) -> str:
    return load().hse_last_error(plan).decode()


# ------------------------------------------------------ torch convenience
class Plan:
    """Owns an ``hse_plan``; methods take torch CUDA float64 tensors."""

    def __init__(self, kernel_mask, box=(1.0, 1.0, 1.0), xi=0.0, rc=0.0, P=0, tol=0.0, precision=HSE_FP64, M=None):
        self.handle = hse_plan_create(kernel_mask, box, xi, rc, P, tol, precision)
        if M is not None:
            hse_plan_set_grid(self.handle, M)
        self.params = hse_plan_get_params(self.handle)

    def set_rc64(self, rc64):
        hse_plan_set_rc64(self.handle, rc64)
        self.params = hse_plan_get_params(self.handle)

    def set_rcmid(self, rcmid):
        hse_plan_set_rcmid(self.handle, rcmid)
        self.params = hse_plan_get_params(self.handle)

    def set_grid(self, M):
        hse_plan_set_grid(self.handle, M)
        self.params = hse_plan_get_params(self.handle)

    def set_fft(self, mode):
        hse_plan_set_fft(self.handle, mode)
        self.params = hse_plan_get_params(self.handle)

    @staticmethod
    def _ptr(t):
        if t is None:
            return None
        import torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected a contiguous float64 CUDA tensor")
        return t.data_ptr()

    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def eval(self, src, strengths, tgt=None, out=None):
        import torch
        n_src = src.shape[1]
        n_tgt = n_src if tgt is None else tgt.shape[1]
        if out is None:
            out = torch.empty((3, n_tgt), dtype=torch.float64, device=src.device)
        hse_eval(self.handle, n_src, self._ptr(src), self._ptr(strengths), n_tgt, self._ptr(tgt), self._ptr(out),
                 self._stream())
        return out

    def eval_parts(self, src, strengths, tgt=None, real=True, fourier=True):
        import torch
        n_src = src.shape[1]
        n_tgt = n_src if tgt is None else tgt.shape[1]
        ur = torch.empty((3, n_tgt), dtype=torch.float64, device=src.device) if real else None
        uf = torch.empty((3, n_tgt), dtype=torch.float64, device=src.device) if fourier else None
        hse_eval_parts(self.handle, n_src, self._ptr(src), self._ptr(strengths), n_tgt, self._ptr(tgt),
                       None if ur is None else ur.data_ptr(), None if uf is None else uf.data_ptr(), self._stream())
        return ur, uf

    def cell_list(self, pos):
        import torch
        n = pos.shape[1]
        nc = self.params["ncell"]
        cid = torch.empty(n, dtype=torch.int32, device=pos.device)
        perm = torch.empty(n, dtype=torch.int32, device=pos.device)
        start = torch.empty(nc[0] * nc[1] * nc[2] + 1, dtype=torch.int32, device=pos.device)
        hse_cell_list(self.handle, n, self._ptr(pos), cid.data_ptr(), perm.data_ptr(), start.data_ptr(),
                      self._stream())
        return cid, perm, start

    def neighbor_counts(self, src, tgt=None):
        import torch
        n_src = src.shape[1]
        n_tgt = n_src if tgt is None else tgt.shape[1]
        a = torch.empty(n_tgt, dtype=torch.int32, device=src.device)
        b = torch.empty(n_tgt, dtype=torch.int32, device=src.device)
        hse_neighbor_counts(self.handle, n_src, self._ptr(src), n_tgt, self._ptr(tgt), a.data_ptr(), b.data_ptr(),
                            self._stream())
        return a, b

    def spread_grids(self, src, strengths):
        import torch
        nc = hse_spread_grids(self.handle, 0, None, None, None, self._stream())
        Mt = self.params["Mt"]
        g = torch.empty((nc, Mt, Mt, 2 * Mt), dtype=torch.float64, device=src.device)
        hse_spread_grids(self.handle, src.shape[1], self._ptr(src), self._ptr(strengths), g.data_ptr(),
                         self._stream())
        return g

    def set_timing(self, enable=True):
        hse_plan_set_timing(self.handle, enable)

    def set_overlap(self, enable=True):
        hse_plan_set_overlap(self.handle, enable)

    def set_real_residency(self, blocks_per_sm):
        hse_plan_set_real_residency(self.handle, blocks_per_sm)

    def set_spread_tile(self, wx, wy, wz):
        hse_plan_set_spread_tile(self.handle, wx, wy, wz)
        self.params = hse_plan_get_params(self.handle)

    def stats(self):
        return hse_get_eval_stats(self.handle)

    def close(self):
        if self.handle is not None:
            hse_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
