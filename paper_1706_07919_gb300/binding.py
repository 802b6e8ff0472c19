"""Thin ctypes binding of include/bie.h.

Module-level functions carry the C names (bie_create, bie_set_geometry, ...) and only marshal
arguments: torch tensors give device pointers and the stream, numpy arrays give host pointers.
Every computation runs in libbie.so; there is no fallback.  Importing this module on a machine
without the built library raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbie.so")

BIE_OK = 0
BIE_ERR_INVALID_ARG = -1
BIE_ERR_CUDA = -2
BIE_ERR_OOM = -3
BIE_ERR_SINGULAR = -4
BIE_ERR_NOT_CONVERGED = -5
BIE_ERR_TIMEOUT = -6
BIE_ERR_STATE = -7
BIE_MODE_FP64 = 0
BIE_MODE_MIXED = 1
BIE_MODE_LEARNED = 2
BIE_MLP_PARAMS = 148738
BIE_FLAG_NOT_CONVERGED = 1
BIE_FLAG_FALLBACK_FP64 = 2
BIE_FLAG_ZERO_PIVOT = 4
BIE_FLAG_ILL_CONDITIONED = 8
BIE_FLAG_FP64_ASSEMBLY = 16
BIE_FLAG_FP32_REFACTOR = 32

EXPORTED = ["bie_last_error", "bie_version", "bie_kernel_launches", "bie_create", "bie_destroy", "bie_set_quadrature",
            "bie_set_geometry", "bie_set_incident_plane_wave", "bie_set_option", "bie_assemble", "bie_solve_frequencies",
            "bie_eval_field", "bie_pulse_spectrum", "bie_synthesize", "bie_synthesize_noalloc", "bie_mlp_set_params",
            "bie_mlp_get_params", "bie_mlp_features", "bie_mlp_forward", "bie_mlp_loss_grad", "bie_mlp_adam_step",
            "bie_mlp_train", "bie_mlp_predict", "bie_get_learned_info", "bie_autotune", "bie_sched_create",
            "bie_sched_destroy", "bie_sched_add", "bie_sched_run", "bie_get_phase_times", "bie_measure_peaks",
            "bie_top_frequencies", "bie_solve_frequencies_multi", "bie_set_geometry_linear",
            "bie_solve_frequencies_async"]


class BieReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("path", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("reserved", ctypes.c_int32), ("backward_err", ctypes.c_double), ("err_est", ctypes.c_double)]


class BieLearnedInfo(ctypes.Structure):
    _fields_ = [("anchors", ctypes.c_int32), ("krylov", ctypes.c_int32), ("krylov_fallback", ctypes.c_int32),
                ("epochs", ctypes.c_int32), ("first_loss", ctypes.c_float), ("last_loss", ctypes.c_float),
                ("train_ms", ctypes.c_double), ("x0_rel_err", ctypes.c_double), ("mean_iters", ctypes.c_double),
                ("max_iters", ctypes.c_double), ("anchors_ms", ctypes.c_double), ("assembly_ms", ctypes.c_double),
                ("predict_ms", ctypes.c_double), ("gmres_ms", ctypes.c_double), ("estimate_ms", ctypes.c_double),
                ("redo_ms", ctypes.c_double)]


class BieTuneResult(ctypes.Structure):
    _fields_ = [("n_bucket", ctypes.c_int32), ("batch", ctypes.c_int32), ("tcgen05", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("us_per_k", ctypes.c_double), ("lu_block", ctypes.c_int32),
                ("lu_panel", ctypes.c_int32), ("lu_tile", ctypes.c_int32)]


class BiePhaseTimes(ctypes.Structure):
    _fields_ = [("assembly_ms", ctypes.c_double), ("factor_ms", ctypes.c_double), ("refine_ms", ctypes.c_double),
                ("reassembly_ms", ctypes.c_double), ("batches", ctypes.c_int32), ("systems", ctypes.c_int32),
                ("reassembled", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BiePeaks(ctypes.Structure):
    _fields_ = [("ffma_tflops", ctypes.c_double), ("dfma_tflops", ctypes.c_double), ("tf32_tflops", ctypes.c_double),
                ("bf16_tflops", ctypes.c_double), ("sm_count", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BieSchedStats(ctypes.Structure):
    _fields_ = [("jobs", ctypes.c_int32), ("workers", ctypes.c_int32), ("wall_ms", ctypes.c_double),
                ("busy_ms", ctypes.c_double)]


class BieError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libbie.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(p)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sigs = {
        "bie_last_error": ([], ctypes.c_char_p),
        "bie_version": ([], ctypes.c_char_p),
        "bie_kernel_launches": ([], ctypes.c_uint64),
        "bie_create": ([ctypes.POINTER(vp), i32, vp], i32),
        "bie_destroy": ([vp], i32),
        "bie_set_quadrature": ([vp, i32, i32], i32),
        "bie_set_geometry": ([vp, vp, i64, vp, i64, vp, vp], i32),
        "bie_set_incident_plane_wave": ([vp, vp], i32),
        "bie_set_option": ([vp, ctypes.c_char_p, dbl], i32),
        "bie_assemble": ([vp, dbl, vp, vp], i32),
        "bie_solve_frequencies": ([vp, vp, i64, i32, vp, vp], i32),
        "bie_eval_field": ([vp, vp, i64, vp, i64, vp, i32, vp], i32),
        "bie_pulse_spectrum": ([vp, vp, i64, i64, vp], i32),
        "bie_synthesize": ([vp, vp, vp, i64, i64, vp, i64, i64, vp, i32], i32),
        "bie_synthesize_noalloc": ([vp, vp, i64, i64, vp, i64, i64, vp, i32, vp], i32),
        "bie_mlp_set_params": ([vp, vp], i32),
        "bie_mlp_get_params": ([vp, vp], i32),
        "bie_mlp_features": ([vp, vp, i64, vp], i32),
        "bie_mlp_forward": ([vp, vp, i64, vp], i32),
        "bie_mlp_loss_grad": ([vp, vp, vp, i64, vp, vp], i32),
        "bie_mlp_adam_step": ([vp, vp, dbl], i32),
        "bie_mlp_train": ([vp, vp, i64, vp, i32, vp], i32),
        "bie_mlp_predict": ([vp, vp, i64, vp], i32),
        "bie_get_learned_info": ([vp, vp], i32),
        "bie_autotune": ([vp, vp, i64, ctypes.c_char_p, vp], i32),
        "bie_sched_create": ([ctypes.POINTER(vp), i32, i32, ctypes.c_char_p], i32),
        "bie_sched_destroy": ([vp], i32),
        "bie_sched_add": ([vp, vp, i64, vp, i64, vp, vp, vp, vp, i64, i32, vp, vp, vp], i32),
        "bie_sched_run": ([vp, vp], i32),
        "bie_get_phase_times": ([vp, vp], i32),
        "bie_measure_peaks": ([i32, vp], i32),
        "bie_top_frequencies": ([vp, vp, i64, i64, i64, vp], i32),
        "bie_solve_frequencies_multi": ([vp, vp, i64, vp, i64, i32, vp, vp], i32),
        "bie_set_geometry_linear": ([vp, vp, i64, vp, i64, vp, vp], i32),
        "bie_solve_frequencies_async": ([vp, vp, i64, i32, vp, vp], i32),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != BIE_OK:
        raise BieError(rc, load().bie_last_error().decode())


def _hp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dp(t) -> int:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


# ---------------------------------------------------------------- C names, marshalling only ----
def bie_last_error() -> str:
    return load().bie_last_error().decode()


def bie_version() -> str:
    return load().bie_version().decode()


def bie_kernel_launches() -> int:
    return int(load().bie_kernel_launches())


def bie_create(device: int = 0, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().bie_create(ctypes.byref(h), device, stream))
    return h.value


def bie_destroy(ctx: int) -> None:
    _check(load().bie_destroy(ctx))


def bie_set_quadrature(ctx: int, ng: int, ng_near: int) -> None:
    _check(load().bie_set_quadrature(ctx, ng, ng_near))


def bie_set_geometry(ctx: int, nodes, elems, normals, bc) -> None:
    nodes = np.ascontiguousarray(nodes, np.float64)
    elems = np.ascontiguousarray(elems, np.int32)
    bc = np.ascontiguousarray(bc, np.uint8)
    nrm = None if normals is None else np.ascontiguousarray(normals, np.float64)
    _check(load().bie_set_geometry(ctx, _hp(nodes), nodes.shape[0], _hp(elems), elems.shape[0],
                                   None if nrm is None else _hp(nrm), _hp(bc)))


def bie_set_geometry_linear(ctx: int, nodes, elems, normals, bc) -> None:
    nodes = np.ascontiguousarray(nodes, np.float64)
    elems = np.ascontiguousarray(elems, np.int32)
    if elems.ndim != 2 or elems.shape[1] != 3:
        raise ValueError("linear elements are [E][3]")
    bc = np.ascontiguousarray(bc, np.uint8)
    nrm = None if normals is None else np.ascontiguousarray(normals, np.float64)
    _check(load().bie_set_geometry_linear(ctx, _hp(nodes), nodes.shape[0], _hp(elems), elems.shape[0],
                                          None if nrm is None else _hp(nrm), _hp(bc)))


def bie_set_incident_plane_wave(ctx: int, direction) -> None:
    d = np.ascontiguousarray(direction, np.float64)
    _check(load().bie_set_incident_plane_wave(ctx, _hp(d)))


def bie_set_option(ctx: int, name: str, value: float) -> None:
    _check(load().bie_set_option(ctx, name.encode(), float(value)))


def bie_assemble(ctx: int, k: float, A, b) -> None:
    _check(load().bie_assemble(ctx, float(k), _dp(A), _dp(b)))


def bie_solve_frequencies(ctx: int, k, mode: int, surf_out, reports: bool = True):
    k = np.ascontiguousarray(k, np.float64)
    rep = (BieReport * max(1, k.shape[0]))() if reports else None
    _check(load().bie_solve_frequencies(ctx, _hp(k), k.shape[0], mode, _dp(surf_out),
                                        ctypes.cast(rep, ctypes.c_void_p) if rep is not None else None))
    return list(rep)[: k.shape[0]] if rep is not None else None


class PendingReports:
    """Reports of a stream-ordered solve: the host array that the library fills in stream order,
    with an event recorded on the context's stream after the call.  `reports()` waits for that
    event; dropping the object also waits for it first, so that the array outlives the library's
    write into it."""

    def __init__(self, arr, n: int, event):
        self._arr, self._n, self._ev = arr, n, event

    def done(self) -> bool:
        return self._ev.query()

    def reports(self):
        self._ev.synchronize()
        return list(self._arr)[: self._n] if self._arr is not None else None

    def __del__(self):
        try:
            self._ev.synchronize()
        except Exception:
            pass


def bie_solve_frequencies_async(ctx: int, k, mode: int, surf_out, stream, reports: bool = True) -> PendingReports:
    """stream: the torch.cuda.Stream the context was created with."""
    import torch

    k = np.ascontiguousarray(k, np.float64)
    if _dtype_name(surf_out) != "complex128" or (k.shape[0] and _numel(surf_out) % (2 * k.shape[0])):
        raise ValueError("surf_out must be complex128 [Nk][2][N]")
    rep = (BieReport * max(1, k.shape[0]))() if reports else None
    _check(load().bie_solve_frequencies_async(ctx, _hp(k), k.shape[0], mode, _dp(surf_out),
                                              ctypes.cast(rep, ctypes.c_void_p) if rep is not None else None))
    ev = torch.cuda.Event()
    ev.record(stream)
    return PendingReports(rep, k.shape[0], ev)


def bie_solve_frequencies_multi(ctx: int, k, dirs, mode: int, surf_out, reports: bool = True):
    k = np.ascontiguousarray(k, np.float64)
    d = np.ascontiguousarray(np.atleast_2d(dirs), np.float64)
    if d.shape[1] != 3:
        raise ValueError("dirs must be [ndir][3]")
    n = k.shape[0] * d.shape[0]
    if _dtype_name(surf_out) != "complex128" or (k.shape[0] and _numel(surf_out) % (2 * n)):
        raise ValueError("surf_out must be complex128 [Nk][ndir][2][N]")
    rep = (BieReport * max(1, n))() if reports else None
    _check(load().bie_solve_frequencies_multi(ctx, _hp(k), k.shape[0], _hp(d), d.shape[0], mode, _dp(surf_out),
                                              ctypes.cast(rep, ctypes.c_void_p) if rep is not None else None))
    return list(rep)[:n] if rep is not None else None


def bie_eval_field(ctx: int, xobs, k, surf, mode: int, T_out) -> None:
    k = np.ascontiguousarray(k, np.float64)
    if len(xobs.shape) != 2 or xobs.shape[1] != 3 or _dtype_name(xobs) != "float64":
        raise ValueError(f"xobs must be float64 [M][3], got {_dtype_name(xobs)} {tuple(xobs.shape)}")
    if _dtype_name(T_out) != "complex128" or _numel(T_out) != k.shape[0] * xobs.shape[0]:
        raise ValueError(f"T_out must be complex128 with Nk*M = {k.shape[0] * xobs.shape[0]} elements")
    _check(load().bie_eval_field(ctx, _dp(xobs), xobs.shape[0], _hp(k), k.shape[0], _dp(surf), mode, _dp(T_out)))


def bie_pulse_spectrum(ctx: int, s, S_out) -> None:
    if len(s.shape) != 2 or _dtype_name(s) != "float64":
        raise ValueError(f"s must be float64 [P][Nt], got {_dtype_name(s)} {tuple(s.shape)}")
    if _dtype_name(S_out) != "complex128" or _numel(S_out) != s.shape[0] * (s.shape[1] // 2 + 1):
        raise ValueError("S_out must be complex128 [P][Nt/2+1]")
    _check(load().bie_pulse_spectrum(ctx, _dp(s), s.shape[0], s.shape[1], _dp(S_out)))


def _dtype_name(t) -> str:
    return str(t.dtype).split(".")[-1]


def _numel(t) -> int:
    return int(t.numel()) if callable(getattr(t, "numel", None)) else int(np.prod(t.shape))


def _synth_shapes(T, midx, S, Nt: int, out, out_dtype: int) -> None:
    """Argument checks of the synthesis calls (sizes and dtypes only): a short or mistyped output
    would otherwise be written past its end on the device."""
    Nk = midx.shape[0]
    if out_dtype not in (0, 1):
        raise ValueError("out_dtype must be 0 (float64) or 1 (float32)")
    if Nk > 0 and (len(T.shape) != 2 or T.shape[0] != Nk or _dtype_name(T) != "complex128"):
        raise ValueError(f"T must be complex128 [Nk={Nk}][M], got {_dtype_name(T)} {tuple(T.shape)}")
    if len(S.shape) != 2 or S.shape[1] != Nt // 2 + 1 or _dtype_name(S) != "complex128":
        raise ValueError(f"S must be complex128 [P][Nt/2+1={Nt // 2 + 1}], got {_dtype_name(S)} {tuple(S.shape)}")
    want = "float64" if out_dtype == 0 else "float32"
    if _dtype_name(out) != want:
        raise ValueError(f"out must have dtype {want} for out_dtype={out_dtype}, got {_dtype_name(out)}")
    P, M = S.shape[0], T.shape[1]
    if _numel(out) != P * M * Nt:
        raise ValueError(f"out must hold P*M*Nt = {P * M * Nt} elements, got {_numel(out)}")


def bie_synthesize(ctx: int, T, midx, S, Nt: int, out, out_dtype: int) -> None:
    midx = np.ascontiguousarray(midx, np.int64)
    _synth_shapes(T, midx, S, Nt, out, out_dtype)
    _check(load().bie_synthesize(ctx, _dp(T), _hp(midx), midx.shape[0], T.shape[1], _dp(S), S.shape[0], Nt,
                                 _dp(out), out_dtype))


def bie_top_frequencies(ctx: int, S, Nt: int, K: int) -> np.ndarray:
    if len(S.shape) != 2 or S.shape[1] != Nt // 2 + 1 or _dtype_name(S) != "complex128":
        raise ValueError(f"S must be complex128 [P][Nt/2+1={Nt // 2 + 1}]")
    out = np.zeros(max(0, int(K)), np.int64)
    _check(load().bie_top_frequencies(ctx, _dp(S), S.shape[0], int(Nt), int(K), _hp(out)))
    return out


def bie_synthesize_noalloc(T, midx, S, Nt: int, out, out_dtype: int, stream: int | None = None) -> None:
    """Allocation-free synthesis for callers that cannot allocate device memory (see bie.h)."""
    midx = np.ascontiguousarray(midx, np.int64)
    _synth_shapes(T, midx, S, Nt, out, out_dtype)
    _check(load().bie_synthesize_noalloc(_dp(T), _hp(midx), midx.shape[0], T.shape[1], _dp(S), S.shape[0], Nt,
                                         _dp(out), out_dtype, stream))


# ---- learned warm start (not part of the paper's method; see bie.h) ---------------------------
def bie_mlp_set_params(ctx: int, theta) -> None:
    th = np.ascontiguousarray(theta, np.float32)
    if th.shape != (BIE_MLP_PARAMS,):
        raise ValueError(f"expected {BIE_MLP_PARAMS} parameters")
    _check(load().bie_mlp_set_params(ctx, _hp(th)))


def bie_mlp_get_params(ctx: int) -> np.ndarray:
    th = np.zeros(BIE_MLP_PARAMS, np.float32)
    _check(load().bie_mlp_get_params(ctx, _hp(th)))
    return th


def bie_mlp_features(ctx: int, k, phi_out) -> None:
    k = np.ascontiguousarray(np.atleast_1d(k), np.float64)
    _check(load().bie_mlp_features(ctx, _hp(k), k.shape[0], _dp(phi_out)))


def bie_mlp_forward(ctx: int, X, Y_out) -> None:
    _check(load().bie_mlp_forward(ctx, _dp(X), X.shape[0], _dp(Y_out)))


def bie_mlp_loss_grad(ctx: int, X, T, grad_out, loss_out) -> None:
    _check(load().bie_mlp_loss_grad(ctx, _dp(X), _dp(T), X.shape[0],
                                    None if grad_out is None else _dp(grad_out),
                                    None if loss_out is None else _dp(loss_out)))


def bie_mlp_adam_step(ctx: int, grad, lr: float) -> None:
    _check(load().bie_mlp_adam_step(ctx, _dp(grad), float(lr)))


def bie_mlp_train(ctx: int, k, surf, epochs: int) -> np.ndarray:
    k = np.ascontiguousarray(np.atleast_1d(k), np.float64)
    hist = np.zeros(max(1, epochs), np.float32)
    _check(load().bie_mlp_train(ctx, _hp(k), k.shape[0], _dp(surf), int(epochs), _hp(hist)))
    return hist[:epochs]


def bie_mlp_predict(ctx: int, k, x0_out) -> None:
    k = np.ascontiguousarray(np.atleast_1d(k), np.float64)
    _check(load().bie_mlp_predict(ctx, _hp(k), k.shape[0], _dp(x0_out)))


def bie_get_learned_info(ctx: int) -> dict:
    info = BieLearnedInfo()
    _check(load().bie_get_learned_info(ctx, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in BieLearnedInfo._fields_}


def bie_get_phase_times(ctx: int) -> dict:
    pt = BiePhaseTimes()
    _check(load().bie_get_phase_times(ctx, ctypes.byref(pt)))
    return {name: getattr(pt, name) for name, _ in BiePhaseTimes._fields_ if name != "reserved"}


def bie_measure_peaks(device: int = 0) -> dict:
    pk = BiePeaks()
    _check(load().bie_measure_peaks(device, ctypes.byref(pk)))
    return {name: getattr(pk, name) for name, _ in BiePeaks._fields_ if name != "reserved"}


# ---- autotuner and scheduler ------------------------------------------------------------------
def bie_autotune(ctx: int, k, cache_path: str | None = None) -> dict:
    k = np.ascontiguousarray(np.atleast_1d(k), np.float64)
    r = BieTuneResult()
    _check(load().bie_autotune(ctx, _hp(k), k.shape[0], None if cache_path is None else cache_path.encode(),
                               ctypes.byref(r)))
    return {name: getattr(r, name) for name, _ in BieTuneResult._fields_}


def bie_sched_create(device: int = 0, workers: int = 4, tune_cache: str | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().bie_sched_create(ctypes.byref(h), device, workers,
                                   None if tune_cache is None else tune_cache.encode()))
    return h.value


def bie_sched_destroy(sched: int) -> None:
    _check(load().bie_sched_destroy(sched))


class SchedJob:
    """Host arrays kept alive until bie_sched_run has consumed them; reports are read back here."""

    def __init__(self, k):
        self.k = np.ascontiguousarray(k, np.float64)
        self.rep = (BieReport * max(1, self.k.shape[0]))()

    def reports(self):
        return list(self.rep)[: self.k.shape[0]]


def bie_sched_add(sched: int, nodes, elems, normals, bc, direction, k, mode: int, surf_out) -> SchedJob:
    nodes = np.ascontiguousarray(nodes, np.float64)
    elems = np.ascontiguousarray(elems, np.int32)
    bc = np.ascontiguousarray(bc, np.uint8)
    nrm = None if normals is None else np.ascontiguousarray(normals, np.float64)
    d = None if direction is None else np.ascontiguousarray(direction, np.float64)
    job = SchedJob(k)
    jid = ctypes.c_int32()
    _check(load().bie_sched_add(sched, _hp(nodes), nodes.shape[0], _hp(elems), elems.shape[0],
                                None if nrm is None else _hp(nrm), _hp(bc), None if d is None else _hp(d),
                                _hp(job.k), job.k.shape[0], mode, _dp(surf_out),
                                ctypes.cast(job.rep, ctypes.c_void_p), ctypes.byref(jid)))
    job.id = jid.value
    return job


def bie_sched_run(sched: int) -> dict:
    st = BieSchedStats()
    _check(load().bie_sched_run(sched, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in BieSchedStats._fields_}
