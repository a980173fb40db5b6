"""Python binding of libpfire, the GB300 (sm_103a) library for the differentiable
wildfire cellular automaton of arXiv 2502.18738 (PyTorchFire).

Argument marshalling only: every step of the automaton runs in the library's CUDA
kernels. PyTorch supplies device memory and streams. The functions ``pf_*`` mirror the
C ABI of ``include/pfire.h`` one to one (tensors in place of device pointers);
``FireModel`` and ``DiffFire`` are thin conveniences on top of them.

There is no CPU path: if ``libpfire.so`` is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

__all__ = [
    "PFireError", "build", "load", "PF_DISCRETE", "PF_DIFF",
    "pf_create", "pf_destroy", "pf_set_env", "pf_set_wind", "pf_set_wind_async", "pf_wait", "pf_set_params",
    "pf_forward", "pf_advance", "pf_backward", "pf_get_state", "pf_set_state", "pf_ignition_map", "pf_loss_bce",
    "pf_set_tuning", "pf_get_tuning", "pf_memory_stats", "pf_autotune", "pf_autotune_ckpt", "pf_batch_last_stats", "pf_batch_set_direct_cells", "pf_profile_read", "pf_batch_submit", "pf_last_error",
    "pf_version", "pf_loss_bce_noalloc", "PF_NOALLOC_BCE_MAX_N", "FireModel", "DiffFire", "PfJob", "make_job",
    "pf_set_accumulator", "pf_reseed", "pf_backward_dca", "pf_loss_eq10", "pf_arrival_probability",
    "pf_affected_count", "pf_jaccard", "pf_manhattan", "pf_set_slope", "simulate", "WildfireModel",
    "pf_stats", "PfStats", "EXPORTED_SYMBOLS",
]

PF_DISCRETE, PF_DIFF = 0, 1
PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ESTATE, PF_ETIMEOUT = 0, -1, -2, -3, -4, -5
_STATUS = {PF_EINVAL: "PF_EINVAL", PF_ENOMEM: "PF_ENOMEM", PF_ECUDA: "PF_ECUDA",
           PF_ESTATE: "PF_ESTATE", PF_ETIMEOUT: "PF_ETIMEOUT"}

LIB_PATH = _build.LIB

# every extern "C" entry point declared in include/pfire.h
EXPORTED_SYMBOLS = [
    "pf_manhattan", "pf_stats", "pf_create", "pf_destroy", "pf_set_env", "pf_set_wind", "pf_set_params", "pf_forward", "pf_advance",
    "pf_backward", "pf_get_state", "pf_set_state", "pf_ignition_map", "pf_loss_bce", "pf_set_tuning",
    "pf_get_tuning", "pf_profile_read", "pf_batch_submit", "pf_last_error", "pf_version",
    "pf_loss_bce_noalloc", "pf_memory_stats", "pf_autotune", "pf_autotune_ckpt", "pf_batch_last_stats", "pf_batch_set_direct_cells", "pf_set_accumulator", "pf_reseed", "pf_backward_dca", "pf_loss_eq10",
    "pf_arrival_probability", "pf_affected_count", "pf_jaccard", "pf_set_slope", "pf_set_wind_async", "pf_wait",
]
PF_NOALLOC_BCE_MAX_N = 67108864


class PFireError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class PfTuning(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("k", ctypes.c_int), ("K", ctypes.c_int), ("profile", ctypes.c_int),
                ("prep", ctypes.c_int), ("tile_rows", ctypes.c_int), ("tape", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class PfStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("cells", ctypes.c_double * 4), ("near_ties_ignite", ctypes.c_longlong),
                ("near_ties_continue", ctypes.c_longlong)]


class PfBatchStats(ctypes.Structure):
    _fields_ = [("disc_cell_steps", ctypes.c_longlong), ("disc_skipped", ctypes.c_longlong),
                ("diff_cell_steps", ctypes.c_longlong), ("diff_skipped", ctypes.c_longlong),
                ("adj_cell_steps", ctypes.c_longlong), ("adj_skipped", ctypes.c_longlong),
                ("ms_forward", ctypes.c_double), ("ms_adjoint", ctypes.c_double),
                ("ms_kernels_from_start", ctypes.c_double), ("waves", ctypes.c_int), ("direct_jobs", ctypes.c_int),
                ("direct_cell_steps", ctypes.c_longlong), ("ms_direct", ctypes.c_double)]


class PfMemoryStats(ctypes.Structure):
    _fields_ = [("checkpoint_bytes", ctypes.c_longlong), ("segment_bytes", ctypes.c_longlong),
                ("qcache_bytes", ctypes.c_longlong), ("tape_bytes", ctypes.c_longlong),
                ("tape_used_bytes", ctypes.c_longlong), ("tape_launches", ctypes.c_int),
                ("tape_recorded", ctypes.c_int), ("K", ctypes.c_int), ("tape_short", ctypes.c_int),
                ("allocations", ctypes.c_longlong), ("frees", ctypes.c_longlong)]


class PfJob(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("T", ctypes.c_int), ("form", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("run", ctypes.c_uint32), ("fire_id", ctypes.c_uint32),
                ("E", ctypes.c_void_p), ("p_veg", ctypes.c_void_p), ("p_den", ctypes.c_void_p),
                ("V_w", ctypes.c_void_p), ("theta_w", ctypes.c_void_p),
                ("p_h", ctypes.c_float), ("c1", ctypes.c_float), ("c2", ctypes.c_float), ("a", ctypes.c_float),
                ("p_continue", ctypes.c_float), ("l", ctypes.c_float),
                ("S_init", ctypes.c_void_p), ("S_out", ctypes.c_void_p),
                ("dL_da", ctypes.c_void_p), ("grad_params", ctypes.c_void_p),
                ("grad_pveg", ctypes.c_void_p), ("grad_pden", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile libpfire.so for sm_103a (no-op when up to date)."""
    return _build.build(force=force)


def load():
    """Load libpfire.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpfire.so is not built ({LIB_PATH}); call paper_2502_18738_gb300.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i, f, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_uint64
        sig = {
            "pf_create": ([ctypes.POINTER(vp), i, i, i, i, u64, vp], i),
            "pf_destroy": ([vp], None),
            "pf_set_env": ([vp, vp, vp, vp, vp, vp], i),
            "pf_set_wind": ([vp, vp, vp, i], i),
            "pf_set_wind_async": ([vp, vp, vp, i], i),
            "pf_wait": ([vp], i),
            "pf_set_params": ([vp, f, f, f, f, f, f], i),
            "pf_forward": ([vp, vp, i, vp], i),
            "pf_advance": ([vp, i, vp], i),
            "pf_backward": ([vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp], i),
            "pf_get_state": ([vp, ctypes.POINTER(i), vp], i),
            "pf_set_state": ([vp, i, vp], i),
            "pf_ignition_map": ([vp, vp], i),
            "pf_stats": ([vp, ctypes.POINTER(PfStats)], i),
            "pf_loss_bce": ([vp, vp, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_double), vp], i),
            "pf_loss_bce_noalloc": ([vp, vp, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_double), vp], i),
            "pf_set_tuning": ([vp, ctypes.POINTER(PfTuning)], i),
            "pf_get_tuning": ([vp, ctypes.POINTER(PfTuning)], i),
            "pf_memory_stats": ([vp, ctypes.POINTER(PfMemoryStats)], i),
            "pf_autotune": ([vp, vp, i, ctypes.POINTER(PfTuning)], i),
            "pf_autotune_ckpt": ([vp, vp, i, ctypes.POINTER(ctypes.c_int)], i),
            "pf_batch_last_stats": ([ctypes.POINTER(PfBatchStats)], i),
            "pf_batch_set_direct_cells": ([ctypes.c_longlong], i),
            "pf_set_accumulator": ([vp, vp], i),
            "pf_reseed": ([vp, ctypes.c_uint64], i),
            "pf_backward_dca": ([vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp], i),
            "pf_loss_eq10": ([vp, vp, i, i, vp, ctypes.POINTER(ctypes.c_double), vp], i),
            "pf_arrival_probability": ([vp, i, i, i, vp, vp], i),
            "pf_set_slope": ([vp, vp], i),
            "pf_affected_count": ([vp, i, ctypes.c_int64, ctypes.POINTER(ctypes.c_longlong), vp], i),
            "pf_jaccard": ([vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), vp], i),
            "pf_manhattan": ([vp, vp, i, ctypes.c_int64, ctypes.POINTER(ctypes.c_longlong), vp], i),
            "pf_profile_read": ([vp, i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_double), i], i),
            "pf_batch_submit": ([ctypes.POINTER(PfJob), i, vp], i),
            "pf_last_error": ([vp], ctypes.c_char_p),
            "pf_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, h=None):
    if rc != PF_OK:
        msg = load().pf_last_error(h).decode()
        raise PFireError(rc, msg)


def _ptr(t, dtype=None, numel=None, what="tensor"):
    """Device pointer of a CUDA tensor (None -> NULL), after shape/dtype checks."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, dtype, numel, what):
    """Pointer of a host or CUDA tensor (None -> NULL), after shape/dtype checks."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ raw ABI

def pf_version() -> str:
    return load().pf_version().decode()


def pf_last_error(h=None) -> str:
    return load().pf_last_error(h).decode()


def pf_create(H, W, form=PF_DISCRETE, realisations=1, seed=0, stream=None):
    h = ctypes.c_void_p()
    _check(load().pf_create(ctypes.byref(h), int(H), int(W), int(form), int(realisations),
                            int(seed) & 0xFFFFFFFFFFFFFFFF, _stream(stream)))
    return h


def pf_destroy(h):
    if h:
        load().pf_destroy(h)


def pf_set_env(h, H, W, E=None, p_veg=None, p_den=None, V_w=None, theta_w=None):
    n = H * W
    f = torch.float32
    _check(load().pf_set_env(h, _ptr(E, f, n, "E"), _ptr(p_veg, f, n, "p_veg"), _ptr(p_den, f, n, "p_den"),
                             _ptr(V_w, f, n, "V_w"), _ptr(theta_w, f, n, "theta_w")), h)


def pf_set_slope(h, H, W, slope_deg):
    """slope_deg: CUDA FP32 [H][W][3][3] (degrees) or None to use the altitude map again."""
    _check(load().pf_set_slope(h, _ptr(slope_deg, torch.float32, H * W * 9, "slope")), h)


def pf_set_wind(h, H, W, V_w, theta_w, from_step):
    n = H * W
    _check(load().pf_set_wind(h, _ptr(V_w, torch.float32, n, "V_w"), _ptr(theta_w, torch.float32, n, "theta_w"),
                              int(from_step)), h)


def pf_set_wind_async(h, H, W, V_w, theta_w, from_step):
    """V_w / theta_w: FP32 H*W tensors in host memory (pinned, for the copy to overlap the
    run) or on the device. They must stay alive and unchanged until the next pf_wait,
    pf_backward or pf_destroy returns."""
    n = H * W
    _check(load().pf_set_wind_async(h, _hptr(V_w, torch.float32, n, "V_w"),
                                    _hptr(theta_w, torch.float32, n, "theta_w"), int(from_step)), h)


def pf_wait(h):
    _check(load().pf_wait(h), h)


def pf_set_params(h, p_h, c1, c2, a, p_continue, l=30.0):
    _check(load().pf_set_params(h, p_h, c1, c2, a, p_continue, l), h)


def pf_forward(h, S_init, T, S_out=None):
    _check(load().pf_forward(h, _ptr(S_init, torch.uint8, None, "S_init"), int(T), _ptr(S_out, None, None, "S_out")), h)
    return S_out


def pf_advance(h, T, S_out=None):
    _check(load().pf_advance(h, int(T), _ptr(S_out, None, None, "S_out")), h)
    return S_out


def pf_backward(h, dL_da=None, dL_db=None, grad_pveg=None, grad_pden=None):
    g = (ctypes.c_double * 4)()
    f = torch.float32
    _check(load().pf_backward(h, _ptr(dL_da, f, None, "dL_da"), _ptr(dL_db, f, None, "dL_db"), g,
                              _ptr(grad_pveg, f, None, "grad_pveg"), _ptr(grad_pden, f, None, "grad_pden")), h)
    return [g[0], g[1], g[2], g[3]]


def pf_get_state(h, S=None) -> int:
    step = ctypes.c_int()
    _check(load().pf_get_state(h, ctypes.byref(step), _ptr(S, None, None, "S")), h)
    return step.value


def pf_set_state(h, step, S):
    _check(load().pf_set_state(h, int(step), _ptr(S, None, None, "S")), h)


def pf_stats(h) -> dict:
    """State counts and discrete near-tie counts of a context (see include/pfire.h)."""
    st = PfStats()
    _check(load().pf_stats(h, ctypes.byref(st)), h)
    return dict(step=st.step, cells=[st.cells[i] for i in range(4)], near_ties_ignite=st.near_ties_ignite,
                near_ties_continue=st.near_ties_continue)


def pf_ignition_map(h, P_out):
    _check(load().pf_ignition_map(h, _ptr(P_out, torch.float32, None, "P_out")), h)
    return P_out


def pf_loss_bce(a, y, dL_da=None, want_loss=True, stream=None):
    n = a.numel()
    loss = ctypes.c_double()
    _check(load().pf_loss_bce(_ptr(a, torch.float32, n, "a"), _ptr(y, torch.float32, n, "y"), n,
                              _ptr(dL_da, torch.float32, n, "dL_da"),
                              ctypes.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def pf_loss_bce_noalloc(a, y, dL_da=None, want_loss=True, stream=None):
    """pf_loss_bce with its scratch in a static device array (no device allocation)."""
    n = a.numel()
    loss = ctypes.c_double()
    _check(load().pf_loss_bce_noalloc(_ptr(a, torch.float32, n, "a"), _ptr(y, torch.float32, n, "y"), n,
                                      _ptr(dL_da, torch.float32, n, "dL_da"),
                                      ctypes.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def pf_set_tuning(h, kernel=0, k=0, K=0, profile=0, prep=0, tile_rows=0, tape=0):
    """kernel 1 plain / 2 blocked, k steps per blocked launch, K checkpoint interval,
    profile, prep 1 materialised q / 2 q recomputed in the step kernels, tile_rows of the
    discrete blocked kernel, tape 1 to recompute every segment; 0 = automatic."""
    t = PfTuning(kernel, k, K, profile, prep, tile_rows, tape)
    _check(load().pf_set_tuning(h, ctypes.byref(t)), h)


def pf_get_tuning(h) -> dict:
    t = PfTuning()
    _check(load().pf_get_tuning(h, ctypes.byref(t)), h)
    return t.as_dict()


def pf_memory_stats(h) -> dict:
    """Device memory of the gradient path (checkpoints, segment buffer, q cache, tile
    tape) and how much of the tape the last taped forward used."""
    st = PfMemoryStats()
    _check(load().pf_memory_stats(h, ctypes.byref(st)), h)
    return {name: getattr(st, name) for name, _ in st._fields_}


def pf_autotune(h, S_init, T_probe) -> dict:
    """Time the candidate launch configurations on a T_probe-step forward from S_init
    and keep the fastest; returns the resulting tuning."""
    t = PfTuning()
    _check(load().pf_autotune(h, _ptr(S_init, torch.uint8, None, "S_init"), int(T_probe), ctypes.byref(t)), h)
    return t.as_dict()


def pf_autotune_ckpt(h, S_init, T) -> int:
    """Time forward + adjoint of T steps for the candidate checkpoint intervals and keep
    the fastest (0 = the memory rule); returns it."""
    K = ctypes.c_int(0)
    _check(load().pf_autotune_ckpt(h, _ptr(S_init, torch.uint8, None, "S_init"), int(T), ctypes.byref(K)), h)
    return K.value


def pf_set_accumulator(h, acc):
    """acc: CUDA FP32 tensor [R][H][W] (kept alive by the caller), or None."""
    _check(load().pf_set_accumulator(h, _ptr(acc, torch.float32, None, "acc")), h)


def pf_reseed(h, seed):
    _check(load().pf_reseed(h, int(seed) & (2**64 - 1)), h)


def pf_backward_dca(h, dL_dacc, step_mask=None, grad_pveg=None, grad_pden=None):
    """Gradient of a loss of the accumulator; step_mask: host bool/uint8 array over the
    steps run (None: all). Returns the 4 parameter gradients (p_h, c1, c2, a)."""
    g4 = (ctypes.c_double * 4)()
    m = None
    if step_mask is not None:
        import numpy as np
        mk = np.ascontiguousarray(np.asarray(step_mask).astype(np.uint8))
        m = mk.ctypes.data_as(ctypes.c_void_p)
    _check(load().pf_backward_dca(h, _ptr(dL_dacc, torch.float32, None, "dL_dacc"), m, g4,
                                  _ptr(grad_pveg, torch.float32, None, "grad_pveg"),
                                  _ptr(grad_pden, torch.float32, None, "grad_pden")), h)
    return list(g4)


def pf_loss_eq10(yhat, y, dL_dyhat=None, want_loss=True, stream=None):
    """Eq. 10 on one map (CUDA FP32 [H][W] tensors); returns the loss (or None)."""
    H, W = yhat.shape
    loss = ctypes.c_double(0.0)
    _check(load().pf_loss_eq10(_ptr(yhat, torch.float32, H * W, "yhat"), _ptr(y, torch.float32, H * W, "y"), H, W,
                               _ptr(dL_dyhat, torch.float32, H * W, "dL_dyhat"),
                               ctypes.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def pf_arrival_probability(S, P_out=None, stream=None):
    """S: CUDA uint8 [R][H][W]; returns FP32 [H][W] fraction of realisations affected."""
    R, H, W = S.shape
    P_out = torch.empty((H, W), dtype=torch.float32, device="cuda") if P_out is None else P_out
    _check(load().pf_arrival_probability(_ptr(S, torch.uint8, R * H * W, "S"), R, H, W,
                                         _ptr(P_out, torch.float32, H * W, "P_out"), _stream(stream)))
    return P_out


def pf_affected_count(S, stream=None):
    """S: CUDA uint8 [R][...]; returns a list of R affected-cell counts."""
    R = S.shape[0]
    n = S.numel() // R
    out = (ctypes.c_longlong * R)()
    _check(load().pf_affected_count(_ptr(S, torch.uint8, None, "S"), R, n, out, _stream(stream)))
    return [int(v) for v in out]


def pf_jaccard(A, B, stream=None):
    """Eq. 11 between the affected sets of two CUDA uint8 state maps of equal size."""
    out = ctypes.c_double(0.0)
    _check(load().pf_jaccard(_ptr(A, torch.uint8, None, "A"), _ptr(B, torch.uint8, A.numel(), "B"), A.numel(),
                             ctypes.byref(out), _stream(stream)))
    return out.value


def pf_manhattan(SA, SB, stream=None) -> int:
    """Eq. 12 between two runs, each a series of T states (uint8 CUDA tensors [T][H][W],
    the state after each step of one realisation), computed on the device."""
    if SA.shape != SB.shape or SA.dim() < 2:
        raise ValueError("pf_manhattan: SA and SB must be [T][...] tensors of one shape")
    T = SA.shape[0]
    HW = SA.numel() // T
    out = ctypes.c_longlong()
    _check(load().pf_manhattan(_ptr(SA, torch.uint8, None, "SA"), _ptr(SB, torch.uint8, None, "SB"), int(T),
                               int(HW), ctypes.byref(out), _stream(stream)))
    return int(out.value)


def pf_profile_read(h, reset=False) -> dict:
    """{kernel kind: (launches, cell_steps, device ms, skipped cell_steps)} since the last
    reset; skipped = cell-steps of quiescent tiles the blocked kernels did not compute."""
    n = 16
    kinds = (ctypes.c_char_p * n)()
    launches = (ctypes.c_longlong * n)()
    steps = (ctypes.c_longlong * n)()
    skipped = (ctypes.c_longlong * n)()
    ms = (ctypes.c_double * n)()
    m = load().pf_profile_read(h, n, kinds, launches, steps, skipped, ms, int(bool(reset)))
    if m < 0:
        _check(m, h)
    return {kinds[i].decode(): (int(launches[i]), int(steps[i]), float(ms[i]), int(skipped[i])) for i in range(m)}


def make_job(S_init, T, S_out=None, form=PF_DISCRETE, seed=0, run=0, fire_id=0, E=None, p_veg=None, p_den=None,
             V_w=None, theta_w=None, p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0,
             dL_da=None, grad_params=None, grad_pveg=None, grad_pden=None):
    """A PfJob over CUDA tensors (S_init uint8 [H][W]); allocates S_out if not given
    (uint8 [H][W] discrete, FP32 [2][H][W] differentiable). Returns (job, S_out); the job
    keeps references to every tensor it points into."""
    H, W = S_init.shape
    if S_out is None:
        S_out = (torch.empty((H, W), dtype=torch.uint8, device="cuda") if form == PF_DISCRETE
                 else torch.empty((2, H, W), dtype=torch.float32, device="cuda"))
    n = H * W
    j = PfJob()
    j.H, j.W, j.T, j.form = H, W, int(T), int(form)
    j.seed, j.run, j.fire_id = int(seed) & (2**64 - 1), int(run), int(fire_id)
    for name, t in (("E", E), ("p_veg", p_veg), ("p_den", p_den), ("V_w", V_w), ("theta_w", theta_w)):
        p = _ptr(t, torch.float32, n, name)
        setattr(j, name, p.value if p is not None else None)
    j.p_h, j.c1, j.c2, j.a, j.p_continue, j.l = p_h, c1, c2, a, p_continue, l
    j.S_init = _ptr(S_init, torch.uint8, n, "S_init").value
    j.S_out = _ptr(S_out, torch.uint8 if form == PF_DISCRETE else torch.float32,
                   n * (1 if form == PF_DISCRETE else 2), "S_out").value
    if dL_da is not None and grad_params is None:
        grad_params = torch.zeros(4, dtype=torch.float64, device="cuda")
    for name, t, dt, nn in (("dL_da", dL_da, torch.float32, n), ("grad_params", grad_params, torch.float64, 4),
                            ("grad_pveg", grad_pveg, torch.float32, n), ("grad_pden", grad_pden, torch.float32, n)):
        p = _ptr(t, dt, nn, name)
        setattr(j, name, p.value if p is not None else None)
    j._keep = (S_init, S_out, E, p_veg, p_den, V_w, theta_w, dL_da, grad_params, grad_pveg, grad_pden)
    j.grads = grad_params  # device double[4] (p_h, c1, c2, a) after pf_batch_submit, or None
    return j, S_out


def pf_batch_submit(jobs, stream=None):
    arr = (PfJob * len(jobs))(*jobs)
    _check(load().pf_batch_submit(arr, len(jobs), _stream(stream)))


def pf_batch_set_direct_cells(min_cells: int):
    """Jobs of pf_batch_submit with H * W >= min_cells run through contexts of their own."""
    _check(load().pf_batch_set_direct_cells(int(min_cells)))


def pf_batch_last_stats() -> dict:
    """Cell-steps computed / skipped and device ms of this thread's last pf_batch_submit."""
    st = PfBatchStats()
    _check(load().pf_batch_last_stats(ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in st._fields_}


# ------------------------------------------------------------- conveniences

class FireModel:
    """One libpfire context (an H x W grid, one form) on the current CUDA stream."""

    def __init__(self, H, W, form=PF_DISCRETE, realisations=1, seed=0, stream=None):
        self.H, self.W, self.form, self.R = int(H), int(W), int(form), int(realisations)
        self.h = pf_create(H, W, form, realisations, seed, stream)

    def close(self):
        if getattr(self, "h", None):
            pf_destroy(self.h)
            self.h = None

    __del__ = close

    def set_env(self, E=None, p_veg=None, p_den=None, V_w=None, theta_w=None):
        pf_set_env(self.h, self.H, self.W, E, p_veg, p_den, V_w, theta_w)

    def set_wind(self, V_w, theta_w, from_step):
        pf_set_wind(self.h, self.H, self.W, V_w, theta_w, from_step)

    def set_wind_async(self, V_w, theta_w, from_step):
        """pf_set_wind_async; the model keeps V_w / theta_w alive until the next wait()."""
        pf_set_wind_async(self.h, self.H, self.W, V_w, theta_w, from_step)
        self.__dict__.setdefault("_uploads", []).append((V_w, theta_w))

    def wait(self):
        pf_wait(self.h)
        self.__dict__.pop("_uploads", None)

    def set_slope(self, slope_deg=None):
        pf_set_slope(self.h, self.H, self.W, slope_deg)

    def set_params(self, p_h, c1, c2, a, p_continue, l=30.0):
        pf_set_params(self.h, p_h, c1, c2, a, p_continue, l)

    def set_tuning(self, **kw):
        pf_set_tuning(self.h, **kw)

    def autotune(self, S_init, T_probe=64):
        return pf_autotune(self.h, S_init, T_probe)

    def autotune_ckpt(self, S_init, T):
        return pf_autotune_ckpt(self.h, S_init, T)

    def set_accumulator(self, acc=None):
        """Attach (or, with None, detach) an FP32 [R][H][W] accumulator tensor; returns it."""
        self._acc = acc
        pf_set_accumulator(self.h, acc)
        return acc

    def reseed(self, seed):
        pf_reseed(self.h, seed)

    def backward_dca(self, dL_dacc, step_mask=None, per_cell=True):
        gpv = gpd = None
        if per_cell:
            gpv = torch.empty((self.H, self.W), dtype=torch.float32, device="cuda")
            gpd = torch.empty_like(gpv)
        g = pf_backward_dca(self.h, dL_dacc, step_mask, gpv, gpd)
        return g, gpv, gpd

    def _out(self):
        if self.form == PF_DISCRETE:
            return torch.empty((self.R, self.H, self.W), dtype=torch.uint8, device="cuda")
        return torch.empty((2, self.H, self.W), dtype=torch.float32, device="cuda")

    def forward(self, S_init, T, out=None):
        out = self._out() if out is None else out
        return pf_forward(self.h, S_init, T, out)

    def advance(self, T, out=None):
        out = self._out() if out is None else out
        return pf_advance(self.h, T, out)

    def backward(self, dL_da=None, dL_db=None, per_cell=True):
        gpv = gpd = None
        if per_cell:
            gpv = torch.empty((self.H, self.W), dtype=torch.float32, device="cuda")
            gpd = torch.empty_like(gpv)
        g = pf_backward(self.h, dL_da, dL_db, gpv, gpd)
        self.__dict__.pop("_uploads", None)  # pf_backward waited for the uploads
        return g, gpv, gpd

    def state(self):
        out = self._out()
        step = pf_get_state(self.h, out)
        return step, out

    def set_state(self, step, S):
        pf_set_state(self.h, step, S)

    def ignition_map(self):
        P = torch.empty((self.R if self.form == PF_DISCRETE else 1, self.H, self.W), dtype=torch.float32,
                        device="cuda")
        return pf_ignition_map(self.h, P)

    def stats(self) -> dict:
        return pf_stats(self.h)


class DiffFire(torch.autograd.Function):
    """Differentiable forward through pf_forward and adjoint through pf_backward.

    ``a_T, b_T = DiffFire.apply(model, S_init, T, params4, p_veg, p_den)`` where params4 =
    (p_h, c1, c2, a) as a float64 tensor (CPU or CUDA) and p_veg / p_den are H x W float32
    CUDA tensors. The model's other inputs (E, wind epochs, p_continue, l) are held
    fixed."""

    @staticmethod
    def forward(ctx, model: FireModel, S_init, T, params4, p_veg, p_den, p_continue=0.3, l=30.0,
                E=None, V_w=None, theta_w=None):
        p = [float(x) for x in params4.detach().cpu().tolist()]
        model.set_env(E, p_veg.detach().contiguous(), p_den.detach().contiguous(), V_w, theta_w)
        model.set_params(p[0], p[1], p[2], p[3], p_continue, l)
        out = model.forward(S_init, T)
        ctx.model = model
        ctx.params_dtype, ctx.params_device = params4.dtype, params4.device
        return out[0].clone(), out[1].clone()

    @staticmethod
    def backward(ctx, ga, gb):
        ga = None if ga is None else ga.contiguous().float()
        gb = None if gb is None else gb.contiguous().float()
        g, gpv, gpd = ctx.model.backward(ga, gb, per_cell=True)
        g4 = torch.tensor(g, dtype=ctx.params_dtype, device=ctx.params_device)
        return None, None, None, g4, gpv, gpd, None, None, None, None, None


def simulate(S_init, T, E=None, p_veg=None, p_den=None, V_w=None, theta_w=None, slope=None, realisations=1, seed=0,
             p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0, kernel=0):
    """Run the discrete form for T steps (Sec. 2.2): S_init CUDA uint8 [H][W] (or
    [R][H][W]); fields CUDA FP32 [H][W] (None: neutral), slope the optional
    [H][W][3][3] tensor in degrees. Returns the uint8 state [R][H][W] after T steps."""
    if S_init.dim() == 2:
        S_init = S_init.expand(realisations, *S_init.shape).contiguous()
    R, H, W = S_init.shape
    m = FireModel(H, W, PF_DISCRETE, R, seed=seed)
    try:
        m.set_env(E, p_veg, p_den, V_w, theta_w)
        if slope is not None:
            m.set_slope(slope)
        m.set_params(p_h, c1, c2, a, p_continue, l)
        if kernel:
            m.set_tuning(kernel=kernel)
        return m.forward(S_init, T)
    finally:
        m.close()


class WildfireModel:
    """The paper's model object (Sec. 2.1 inputs and outputs, the calls of Alg. 1) over
    the discrete form: ``compute(attach)`` advances one step, ``reset(seed)`` returns to
    the initial fire, ``state`` is the two-channel (burning, burned) map, ``accumulator``
    holds p_ignite of the newly ignited cells, ``ignition_map()`` is p_ignite, and
    ``backward(dL_dacc)`` returns the parameter gradients through the attached steps.

    Inputs: CUDA tensors H x W (wind velocity m/s, wind direction degrees counter-
    clockwise from East, canopy p_veg, density p_den), the slope as H x W x 3 x 3 degrees
    or an altitude map E, the initial fire as an H x W boolean (burning) map, an optional
    non-burnable mask, and the five parameters."""

    def __init__(self, initial_fire, wind_velocity=None, wind_direction=None, slope=None, altitude=None,
                 canopy=None, density=None, non_burnable=None, p_h=0.58, c1=0.045, c2=0.131, a=0.078,
                 p_continue=0.3, cell_size=30.0, seed=0):
        H, W = initial_fire.shape
        S = torch.ones((H, W), dtype=torch.uint8, device="cuda")
        if non_burnable is not None:
            S[non_burnable.bool()] = 0
        S[initial_fire.bool()] = 2
        self.S_init = S[None].contiguous()
        self.H, self.W = H, W
        self.params = dict(p_h=p_h, c1=c1, c2=c2, a=a, p_continue=p_continue, l=cell_size)
        self.m = FireModel(H, W, PF_DISCRETE, 1, seed=seed)
        self.fields = (altitude, canopy, density)
        self.m.set_env(altitude, canopy, density, wind_velocity, wind_direction)
        if slope is not None:
            self.m.set_slope(slope.contiguous())
        self.m.set_params(**self.params)
        self.accumulator = self.m.set_accumulator(torch.zeros((1, H, W), dtype=torch.float32, device="cuda"))
        self.seed = seed
        self.reset(seed)

    def set_parameters(self, **kw):
        self.params.update(kw)
        self.m.set_params(**self.params)

    def set_wind(self, wind_velocity, wind_direction):
        """Wind for the following steps. Alg. 1 sets it per iteration, before the
        re-simulation from the initial fire; a change after steps were computed starts a
        new wind epoch there and ends the recorded trajectory (call reset before backward)."""
        if self.steps == 0:
            self.m.set_env(*self.fields, wind_velocity, wind_direction)
            self._S = self.m.forward(self.S_init, 0)
        else:
            self.m.set_wind(wind_velocity, wind_direction, self.steps)

    def reset(self, seed=None):
        if seed is not None:
            self.seed = seed
            self.m.reseed(seed)
        self._S = self.m.forward(self.S_init, 0)
        self.steps = 0
        self.attached = []

    def compute(self, attach=False):
        self._S = self.m.advance(1)
        self.attached.append(bool(attach))
        self.steps += 1

    @property
    def state(self):
        """Two-channel boolean map (burning, burned), 2 x H x W."""
        s = self._S[0]
        return torch.stack([s == 2, s == 3])

    def ignition_map(self):
        return self.m.ignition_map()[0]

    def backward(self, dL_dacc):
        """Gradients (p_h, c1, c2, a) of a loss whose gradient with respect to the
        accumulator is dL_dacc (H x W); only the attached steps carry gradient."""
        g, _, _ = self.m.backward_dca(dL_dacc.reshape(1, self.H, self.W).contiguous().float(),
                                      step_mask=self.attached, per_cell=False)
        return g
