"""Python binding of libkstap (include/kstap.h): argument marshalling only.

Every step of the Kron-STAP path runs in the CUDA kernels of libkstap.so; this
module converts torch tensors / ints to the C ABI's plain pointers and sizes.
There is no CPU fallback: if the shared library is missing or fails to load,
importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkstap.so")

KSTAP_OK = 0
KSTAP_WARN_NOCONV = 1
STATUS = {1: "KSTAP_WARN_NOCONV", 0: "KSTAP_OK", -1: "KSTAP_EINVAL", -2: "KSTAP_ENOMEM", -3: "KSTAP_ECUDA",
          -4: "KSTAP_EAGAIN", -5: "KSTAP_ETIMEOUT", -6: "KSTAP_ENOTFOUND"}

EXPORTED = ["kstap_create", "kstap_fit_project", "kstap_detect", "kstap_destroy",
            "kstap_last_error", "kstap_workspace_bytes", "kstap_set_profiling",
            "kstap_kernel_times", "kstap_fit_project_noalloc", "kstap_run_batch",
            "kstap_graph_create", "kstap_graph_launch", "kstap_graph_destroy", "kstap_autotune",
            "kstap_set_tuning", "kstap_serve_config", "kstap_submit", "kstap_poll",
            "kstap_release", "kstap_fit_report", "kstap_device_status", "kstap_lrkron_fit",
            "kstap_change_map", "kstap_serve_batch_cells", "kstap_alu_probe"]
KERNELS = ["frame_scale", "moments", "flipflop", "bfit", "detect", "mgram"]


class KstapParams(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("q", ctypes.c_int), ("r_a", ctypes.c_int),
                ("r_b", ctypes.c_int), ("ring_r", ctypes.c_int), ("ring_a", ctypes.c_int),
                ("guard_r", ctypes.c_int), ("guard_a", ctypes.c_int), ("eps", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("tau", ctypes.c_float), ("precision", ctypes.c_int),
                ("filter", ctypes.c_int)]


class KstapFactors(ctypes.Structure):
    _fields_ = [("UA", ctypes.c_void_p), ("UB_hi", ctypes.c_void_p), ("UB_lo", ctypes.c_void_p),
                ("lamA", ctypes.c_void_p), ("lamB", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("eta", ctypes.c_void_p)]


class KstapFrame(ctypes.Structure):
    _fields_ = [("Y", ctypes.c_void_p), ("H_in", ctypes.c_int), ("W_in", ctypes.c_int),
                ("factors", KstapFactors), ("Tmax", ctypes.c_void_p), ("vidx", ctypes.c_void_p),
                ("map", ctypes.c_void_p), ("T_all", ctypes.c_void_p)]


class KstapTuning(ctypes.Structure):
    _fields_ = [("waves", ctypes.c_int), ("tc", ctypes.c_int), ("lag_store", ctypes.c_int),
                ("ms_per_batch", ctypes.c_float)]


class KstapResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("Tmax", ctypes.c_void_p), ("vidx", ctypes.c_void_p), ("map", ctypes.c_void_p),
                ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]


KSTAP_FRAME_ON_HOST = 1


class KstapError(RuntimeError):
    pass


_lib = None


def lib() -> ctypes.CDLL:
    """Load libkstap.so (built by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise KstapError(f"libkstap.so not built ({LIB_PATH}); run "
                             "python -m paper_1604_03622_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.kstap_create.argtypes = [ctypes.POINTER(KstapParams), P, P, I, Z, P,
                                   ctypes.POINTER(ctypes.c_void_p)]
        L.kstap_fit_project.argtypes = [P, P, I, I, ctypes.POINTER(KstapFactors)]
        L.kstap_detect.argtypes = [P, P, I, I, ctypes.POINTER(KstapFactors), P, P, P, P]
        L.kstap_destroy.argtypes = [P]
        L.kstap_last_error.argtypes = [P]
        L.kstap_last_error.restype = ctypes.c_char_p
        L.kstap_workspace_bytes.argtypes = [ctypes.POINTER(KstapParams), I, I]
        L.kstap_workspace_bytes.restype = Z
        L.kstap_fit_project_noalloc.argtypes = [ctypes.POINTER(KstapParams), P, I, I,
                                                ctypes.POINTER(KstapFactors), P]
        L.kstap_run_batch.argtypes = [P, ctypes.POINTER(KstapFrame), I]
        L.kstap_graph_create.argtypes = [ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.POINTER(KstapFrame)),
                                         ctypes.POINTER(ctypes.c_int), I,
                                         ctypes.POINTER(ctypes.c_void_p)]
        L.kstap_graph_launch.argtypes = [P, P]
        L.kstap_graph_destroy.argtypes = [P]
        L.kstap_autotune.argtypes = [P, ctypes.POINTER(KstapFrame), I, I,
                                     ctypes.POINTER(KstapTuning)]
        L.kstap_set_tuning.argtypes = [P, ctypes.POINTER(KstapTuning)]
        L.kstap_serve_config.argtypes = [P, I, I]
        L.kstap_serve_batch_cells.argtypes = [P, ctypes.c_longlong]
        L.kstap_submit.argtypes = [P, P, I, I, I, ctypes.POINTER(ctypes.c_uint64)]
        L.kstap_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(KstapResult), I]
        L.kstap_release.argtypes = [P, ctypes.c_uint64]
        L.kstap_device_status.argtypes = [P]
        L.kstap_lrkron_fit.argtypes = [P, I, I, I, I, ctypes.c_double, I, P, P,
                                       ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_double), P]
        L.kstap_change_map.argtypes = [P, ctypes.c_longlong, I, I, P, P, P]
        L.kstap_fit_report.argtypes = [P, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong)]
        L.kstap_alu_probe.argtypes = [I, I, I, P, ctypes.POINTER(ctypes.c_double)]
        L.kstap_set_profiling.argtypes = [P, I]
        L.kstap_kernel_times.argtypes = [P, P, P, I]
        for name in ("kstap_create", "kstap_fit_project", "kstap_detect", "kstap_destroy",
                     "kstap_set_profiling", "kstap_kernel_times", "kstap_fit_project_noalloc",
                     "kstap_run_batch", "kstap_graph_create", "kstap_graph_launch",
                     "kstap_graph_destroy", "kstap_autotune", "kstap_set_tuning",
                     "kstap_serve_config", "kstap_submit", "kstap_poll", "kstap_release",
                     "kstap_fit_report", "kstap_device_status", "kstap_lrkron_fit",
                     "kstap_change_map", "kstap_serve_batch_cells", "kstap_alu_probe"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _check(st: int, ctx: Optional[int] = None) -> None:
    if st != KSTAP_OK:
        msg = lib().kstap_last_error(ctx).decode()
        raise KstapError(f"{STATUS.get(st, st)}: {msg}")


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


PRECISION = {"fp32": 0, "fp16x3": 1, "bf16x3": 2}
FILTER = {"kron": 0, "classical": 1}


def make_params(p, q, r_a, r_b, ring_r, ring_a, guard_r, guard_a, tau, eps=0.0,
                max_iter=0, precision="fp32", filter="kron") -> KstapParams:
    return KstapParams(p, q, r_a, r_b, ring_r, ring_a, guard_r, guard_a, float(eps),
                       int(max_iter), float(tau), PRECISION[precision], FILTER[filter])


def kstap_create(params: KstapParams, bank_a, bank_b, V: int, hbm_budget_bytes: int = 0,
                 stream: int = 0) -> int:
    """bank_a (V x p), bank_b (V x q): complex64 device tensors.  Returns ctx."""
    out = ctypes.c_void_p()
    _check(lib().kstap_create(ctypes.byref(params), _ptr(bank_a), _ptr(bank_b), V,
                              hbm_budget_bytes, stream or None, ctypes.byref(out)))
    return out.value


def make_factors(UA, UB_hi, UB_lo, lamA=None, lamB=None, iters=None, eta=None) -> KstapFactors:
    return KstapFactors(_ptr(UA), _ptr(UB_hi), _ptr(UB_lo), _ptr(lamA), _ptr(lamB),
                        _ptr(iters), _ptr(eta))


def kstap_fit_project(ctx: int, Y, H_in: int, W_in: int, factors: KstapFactors) -> None:
    _check(lib().kstap_fit_project(ctx, _ptr(Y), H_in, W_in, ctypes.byref(factors)), ctx)


def kstap_fit_report(ctx: int):
    """(nonconverged, nonfinite, eig_refined) cell counts of the last fit; waits
    for the stream.  A KSTAP_WARN_NOCONV status is returned in the counts, not
    raised."""
    nc, nf, nr = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    st = lib().kstap_fit_report(ctx, ctypes.byref(nc), ctypes.byref(nf), ctypes.byref(nr))
    if st != KSTAP_WARN_NOCONV:
        _check(st, ctx)
    return int(nc.value), int(nf.value), int(nr.value)


def kstap_lrkron_fit(X, r_a: int = 1, eps: float = 1e-6, max_iter: int = 100, A_out=None,
                     B_out=None, stream: int = 0):
    """One large-covariance LR-Kron fit from snapshots X (n, p, q) complex64 on
    the device.  A_out (p, p) and B_out (q, q) are complex64 device tensors
    (allocated with torch when None).  Returns (A_out, B_out, iters, eta)."""
    import torch
    n, p, q = X.shape
    if A_out is None:
        A_out = torch.empty(p, p, dtype=torch.complex64, device=X.device)
    if B_out is None:
        B_out = torch.empty(q, q, dtype=torch.complex64, device=X.device)
    it, et = ctypes.c_int32(), ctypes.c_double()
    _check(lib().kstap_lrkron_fit(_ptr(X), n, p, q, r_a, float(eps), int(max_iter), _ptr(A_out),
                                  _ptr(B_out), ctypes.byref(it), ctypes.byref(et), stream or None))
    return A_out, B_out, int(it.value), float(et.value)


PROBES = {"ffma": 0, "ffma2": 1, "imad64": 2, "dfma": 3}


def kstap_alu_probe(op: str, iters: int, reps: int, stream: int = 0) -> float:
    """Operations per second of one arithmetic pipe (op in PROBES; one FMA or
    multiply-add per lane = one operation); synchronises the stream."""
    out = ctypes.c_double()
    _check(lib().kstap_alu_probe(PROBES[op], int(iters), int(reps), stream, ctypes.byref(out)))
    return float(out.value)


def kstap_change_map(T_all, V: int, K: int, Tmax_k=None, change=None, stream: int = 0):
    """Per-pass maxima and the change map (Sec. 8) from T_all (ncell, K V)
    float32 on the device.  Tmax_k (K, ncell) and change (ncell,) are float32
    device tensors (allocated with torch when None).  Returns (Tmax_k, change)."""
    import torch
    ncell = T_all.shape[0]
    if T_all.shape[1] != K * V or not T_all.is_contiguous():
        raise ValueError("T_all must be a contiguous (ncell, K * V) tensor")
    if Tmax_k is None:
        Tmax_k = torch.empty(K, ncell, dtype=torch.float32, device=T_all.device)
    if change is None:
        change = torch.empty(ncell, dtype=torch.float32, device=T_all.device)
    _check(lib().kstap_change_map(_ptr(T_all), ncell, V, K, _ptr(Tmax_k), _ptr(change),
                                  stream or None))
    return Tmax_k, change


def kstap_device_status(ctx: int) -> None:
    """Raises if a kernel gave up a bounded wait for its tensor-core work."""
    _check(lib().kstap_device_status(ctx), ctx)


def kstap_detect(ctx: int, Y, H_in: int, W_in: int, factors: KstapFactors, Tmax, vidx, map_,
                 T_all=None) -> None:
    _check(lib().kstap_detect(ctx, _ptr(Y), H_in, W_in, ctypes.byref(factors), _ptr(Tmax),
                              _ptr(vidx), _ptr(map_), _ptr(T_all)), ctx)


def kstap_destroy(ctx: int) -> None:
    _check(lib().kstap_destroy(ctx))


def kstap_workspace_bytes(params: KstapParams, H_in: int, W_in: int) -> int:
    return int(lib().kstap_workspace_bytes(ctypes.byref(params), H_in, W_in))


def kstap_last_error(ctx: Optional[int]) -> str:
    return lib().kstap_last_error(ctx).decode()


def kstap_set_profiling(ctx: int, enable: bool) -> None:
    _check(lib().kstap_set_profiling(ctx, 1 if enable else 0), ctx)


def kstap_kernel_times(ctx: int):
    """{kernel name: (total ms, launches)} since profiling was enabled."""
    n = len(KERNELS)
    ms = (ctypes.c_float * n)()
    cnt = (ctypes.c_int32 * n)()
    _check(lib().kstap_kernel_times(ctx, ms, cnt, n), ctx)
    return {KERNELS[k]: (float(ms[k]), int(cnt[k])) for k in range(n)}


def kstap_fit_project_noalloc(params: KstapParams, Y, H_in: int, W_in: int,
                              factors: KstapFactors, stream: int = 0) -> None:
    """Allocation-free fit (no context, static device scratch, <= 32768 cells)."""
    _check(lib().kstap_fit_project_noalloc(ctypes.byref(params), _ptr(Y), H_in, W_in,
                                           ctypes.byref(factors), stream or None))


def make_frame(Y, H_in: int, W_in: int, factors: KstapFactors, Tmax, vidx, map_,
               T_all=None) -> KstapFrame:
    return KstapFrame(_ptr(Y), H_in, W_in, factors, _ptr(Tmax), _ptr(vidx), _ptr(map_),
                      _ptr(T_all))


def kstap_run_batch(ctx: int, frames) -> None:
    arr = (KstapFrame * len(frames))(*frames)
    _check(lib().kstap_run_batch(ctx, arr, len(frames)), ctx)


def kstap_graph_create(ctxs, frames_per_ctx) -> int:
    """One CUDA graph over several contexts' batches (frames_per_ctx[c] for ctxs[c])."""
    n = len(ctxs)
    arrays = [(KstapFrame * len(f))(*f) for f in frames_per_ctx]
    fptrs = (ctypes.POINTER(KstapFrame) * n)(*[ctypes.cast(a, ctypes.POINTER(KstapFrame))
                                                for a in arrays])
    counts = (ctypes.c_int * n)(*[len(f) for f in frames_per_ctx])
    cptrs = (ctypes.c_void_p * n)(*ctxs)
    out = ctypes.c_void_p()
    _check(lib().kstap_graph_create(cptrs, fptrs, counts, n, ctypes.byref(out)))
    return out.value


def kstap_graph_launch(graph: int, stream: int = 0) -> None:
    _check(lib().kstap_graph_launch(graph, stream or None))


def kstap_graph_destroy(graph: int) -> None:
    _check(lib().kstap_graph_destroy(graph))


def kstap_autotune(ctx: int, frames, reps: int = 3) -> KstapTuning:
    arr = (KstapFrame * len(frames))(*frames)
    t = KstapTuning()
    _check(lib().kstap_autotune(ctx, arr, len(frames), reps, ctypes.byref(t)), ctx)
    return t


def kstap_set_tuning(ctx: int, waves: int, tc: int = 0, lag_store: int = 1) -> None:
    t = KstapTuning(waves, tc, lag_store, 0.0)
    _check(lib().kstap_set_tuning(ctx, ctypes.byref(t)), ctx)


def kstap_serve_config(ctx: int, max_batch: int, max_inflight: int) -> None:
    _check(lib().kstap_serve_config(ctx, max_batch, max_inflight), ctx)


def kstap_serve_batch_cells(ctx: int, cells: int) -> None:
    """Work cap of one served batch in cells (<= 0: none; default 1 << 20)."""
    _check(lib().kstap_serve_batch_cells(ctx, int(cells)), ctx)


def kstap_submit(ctx: int, Y, H_in: int, W_in: int, on_host: bool = False) -> int:
    """Queue one frame (torch tensor; pinned host tensor when on_host)."""
    t = ctypes.c_uint64()
    _check(lib().kstap_submit(ctx, _ptr(Y), H_in, W_in, KSTAP_FRAME_ON_HOST if on_host else 0,
                              ctypes.byref(t)), ctx)
    return int(t.value)


def kstap_poll(ctx: int, ticket: int, timeout_us: int = -1):
    """KstapResult when done; None if not ready (timeout_us = 0) or timed out."""
    r = KstapResult()
    st = lib().kstap_poll(ctx, ticket, ctypes.byref(r), timeout_us)
    if st in (-4, -5):
        return None
    _check(st, ctx)
    return r


def kstap_release(ctx: int, ticket: int) -> None:
    _check(lib().kstap_release(ctx, ticket), ctx)
