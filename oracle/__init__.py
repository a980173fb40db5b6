"""Plain FP64 CPU oracle of the wildfire cellular automaton (arXiv 2502.18738).

TEST INFRASTRUCTURE, NOT PRODUCT: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. It shares no code with
the CUDA library: the arithmetic lives in ``pfire_oracle.c`` (plain C, FP64, one loop
per equation) and in ``torch_ref.py`` (an independent FP64 PyTorch-autograd restatement
of the differentiable form). This file only marshals numpy arrays into the C routines
and strings the per-step routines together in time.

Which passage each routine follows:

* ``philox`` / ``cell_draws``: Philox4x32-10 (Salmon et al., SC'11); the two uniform
  draws per cell and step of the data-flow description (Sec. 2.2).
* ``prep``: Eq. 1-5 (slope, propagation probability, wind factor, slope factor, f_p).
* ``step_discrete`` / ``forward_discrete``: Sec. 2.2 transition rules with Eq. 9.
* ``step_diff`` / ``diff_forward``: Eq. 9 with the burning indicator replaced by the
  burning probability (the differentiable mean-field reading of Sec. 2.2).
* ``adjoint_step`` / ``prep_adjoint`` / ``diff_backward``: the chain rule of the above.
* ``bce``: binary cross-entropy of the final burn probability.

Pins: every routine here is checked in ``tests/test_oracle_*.py`` against closed forms,
invariants, symmetries, brute-force enumeration, published Philox test vectors, finite
differences and the independent autograd restatement.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfire_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

C_FP = 1.1486328125  # Eq. 8: the paper's c

P_D = ctypes.POINTER(ctypes.c_double)
P_F = ctypes.POINTER(ctypes.c_float)
P_U8 = ctypes.POINTER(ctypes.c_uint8)
P_U32 = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP on the per-cell loops)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x32_10.argtypes = [P_U32, P_U32, P_U32]
        lib.orc_cell_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, P_D, P_D]
        lib.orc_prep.argtypes = [ctypes.c_int, ctypes.c_int, P_F, P_F, P_F, P_F, P_F, P_F, P_U8,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, P_D]
        lib.orc_step_discrete.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P_U8, P_U8, P_D,
                                          ctypes.c_float, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32, P_D, P_D]
        lib.orc_forward_discrete.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P_U8, P_U8,
                                             P_D, ctypes.c_float, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int]
        lib.orc_step_diff.argtypes = [ctypes.c_int, ctypes.c_int, P_D, P_D, P_D, ctypes.c_double,
                                      P_D, P_D, P_D]
        lib.orc_adjoint_step.argtypes = [ctypes.c_int, ctypes.c_int, P_D, P_D, P_D, ctypes.c_double,
                                         P_D, P_D, P_D, P_D, P_D]
        lib.orc_prep_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, P_F, P_F, P_F, P_F, P_F, P_F, P_U8,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, P_D, P_D, P_D, P_D]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def _ptr(x, ty):
    if x is None:
        return ctypes.cast(None, ty)
    return x.ctypes.data_as(ty)


def _f32(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float32)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _u8(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.uint8)


def f32(v: float) -> float:
    """The FP32 value a parameter takes on the GPU, widened exactly to FP64."""
    return float(np.float32(v))


# ------------------------------------------------------------------ Philox

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c, P_U32), _ptr(k, P_U32), _ptr(out, P_U32))
    return out


def cell_draws(seed: int, run: int, step: int, fire: int, cell: int):
    u0, u1 = ctypes.c_double(), ctypes.c_double()
    _load().orc_cell_draws(seed, run, step, fire, cell, ctypes.byref(u0), ctypes.byref(u1))
    return u0.value, u1.value


# -------------------------------------------------------------------- prep

class Params:
    """The five model parameters plus the cell side l (metres); stored as FP32 values."""

    def __init__(self, p_h, c1, c2, a, p_continue, l=30.0, exact=False):
        r = (lambda v: float(v)) if exact else f32
        self.exact = exact
        self.p_h, self.c1, self.c2, self.a = r(p_h), r(c1), r(c2), r(a)
        self.p_continue, self.l = f32(p_continue), r(l)

    def with_(self, **kw):
        d = dict(p_h=self.p_h, c1=self.c1, c2=self.c2, a=self.a, p_continue=self.p_continue, l=self.l,
                 exact=self.exact)
        d.update(kw)
        return Params(**d)


def prep(H, W, E, p_veg, p_den, V, theta, prm: Params, burnable=None, exact_params=False, slope=None):
    """q[8, H, W] (FP64): f_p(p_propagate) into cell j from its neighbour in direction d.
    slope: the H x W x 3 x 3 slope input in degrees (Sec. 2.1), used instead of E."""
    E, p_veg, p_den, V, theta, slope = map(_f32, (E, p_veg, p_den, V, theta, slope))
    burnable = _u8(burnable)
    q = np.zeros((8, H, W), dtype=np.float64)
    _load().orc_prep(H, W, _ptr(E, P_F), _ptr(slope, P_F), _ptr(p_veg, P_F), _ptr(p_den, P_F), _ptr(V, P_F),
                     _ptr(theta, P_F), _ptr(burnable, P_U8), prm.p_h, prm.c1, prm.c2, prm.a, prm.l,
                     _ptr(q, P_D))
    return q


# ---------------------------------------------------------------- discrete

def step_discrete(S, q, p_continue, seed, step, run0=0, fire=0, return_P=False):
    """One step of R realisations. S: uint8 (H,W) or (R,H,W)."""
    S = np.ascontiguousarray(S, dtype=np.uint8)
    squeeze = S.ndim == 2
    S3 = S[None] if squeeze else S
    R, H, W = S3.shape
    out = np.empty_like(S3)
    P = np.zeros(S3.shape) if return_P else None
    u = np.zeros(S3.shape) if return_P else None
    q = _f64(q)
    _load().orc_step_discrete(H, W, R, _ptr(S3, P_U8), _ptr(out, P_U8), _ptr(q, P_D),
                              ctypes.c_float(p_continue), seed, run0, step, fire,
                              _ptr(P, P_D), _ptr(u, P_D))
    if squeeze:
        out = out[0]
        if return_P:
            P, u = P[0], u[0]
    return (out, P, u) if return_P else out


def forward_discrete(S0, q, p_continue, seed, T, step0=0, run0=0, fire=0):
    S0 = np.ascontiguousarray(S0, dtype=np.uint8)
    squeeze = S0.ndim == 2
    S3 = S0[None] if squeeze else S0
    R, H, W = S3.shape
    out = np.empty_like(S3)
    q = _f64(q)
    _load().orc_forward_discrete(H, W, R, _ptr(S3, P_U8), _ptr(out, P_U8), _ptr(q, P_D),
                                 ctypes.c_float(p_continue), seed, run0, step0, fire, T)
    return out[0] if squeeze else out


def trajectory_discrete(S0, q, p_continue, seed, T, step0=0, run0=0, fire=0):
    """All states S_0..S_T of one realisation, with the per-step P and decisive draws."""
    S = np.ascontiguousarray(S0, dtype=np.uint8)
    states, Ps, us = [S], [], []
    for t in range(T):
        S, P, u = step_discrete(S, q, p_continue, seed, step0 + t, run0, fire, return_P=True)
        states.append(S)
        Ps.append(P)
        us.append(u)
    return states, Ps, us


# ----------------------------------------------------------- differentiable

def diff_init(S0):
    """Continuous initial state from a uint8 state: a = [S in {2,3}], b = [S == 2]."""
    S0 = np.asarray(S0)
    a = ((S0 == 2) | (S0 == 3)).astype(np.float64)
    b = (S0 == 2).astype(np.float64)
    return a, b


def step_diff(a, b, q, p_continue, return_P=False):
    a, b, q = _f64(a), _f64(b), _f64(q)
    H, W = a.shape
    a2, b2 = np.empty_like(a), np.empty_like(b)
    P = np.empty_like(a) if return_P else None
    _load().orc_step_diff(H, W, _ptr(a, P_D), _ptr(b, P_D), _ptr(q, P_D), float(p_continue),
                          _ptr(a2, P_D), _ptr(b2, P_D), _ptr(P, P_D))
    return (a2, b2, P) if return_P else (a2, b2)


def adjoint_step(a, b, q, p_continue, la1, lb1, Gq):
    a, b, q, la1, lb1 = map(_f64, (a, b, q, la1, lb1))
    H, W = a.shape
    la0, lb0 = np.empty_like(a), np.empty_like(a)
    assert Gq.dtype == np.float64 and Gq.flags.c_contiguous
    _load().orc_adjoint_step(H, W, _ptr(a, P_D), _ptr(b, P_D), _ptr(q, P_D), float(p_continue),
                             _ptr(la1, P_D), _ptr(lb1, P_D), _ptr(la0, P_D), _ptr(lb0, P_D),
                             _ptr(Gq, P_D))
    return la0, lb0


def prep_adjoint(H, W, E, p_veg, p_den, V, theta, prm: Params, Gq, burnable=None, slope=None):
    E, p_veg, p_den, V, theta, slope = map(_f32, (E, p_veg, p_den, V, theta, slope))
    burnable = _u8(burnable)
    g4 = np.zeros(4)
    gpv = np.zeros((H, W))
    gpd = np.zeros((H, W))
    Gq = _f64(Gq)
    _load().orc_prep_adjoint(H, W, _ptr(E, P_F), _ptr(slope, P_F), _ptr(p_veg, P_F), _ptr(p_den, P_F), _ptr(V, P_F),
                             _ptr(theta, P_F), _ptr(burnable, P_U8), prm.p_h, prm.c1, prm.c2, prm.a,
                             prm.l, _ptr(Gq, P_D), _ptr(g4, P_D), _ptr(gpv, P_D), _ptr(gpd, P_D))
    return g4, gpv, gpd


def _epoch_of(t, starts):
    e = 0
    for k, s in enumerate(starts):
        if t >= s:
            e = k
    return e


def diff_forward(land, winds, starts, prm: Params, S0, T, keep_states=True):
    """Differentiable forward over T steps. winds[k] = (V, theta) applies from step
    starts[k] (starts[0] == 0). Non-burnable cells (state 0 of S0) get q = 0.
    Returns (a_T, b_T, tape) with tape = list of (a_t, b_t) for t = 0..T-1."""
    H, W = S0.shape
    burn = (np.asarray(S0) != 0).astype(np.uint8)
    qs = {}
    a, b = diff_init(S0)
    tape = []
    for t in range(T):
        e = _epoch_of(t, starts)
        if e not in qs:
            qs.clear()
            V, th = winds[e]
            qs[e] = prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=burn)
        if keep_states:
            tape.append((a, b))
        a, b = step_diff(a, b, qs[e], prm.p_continue)
    return a, b, tape


def diff_backward(land, winds, starts, prm: Params, S0, tape, la_T, lb_T):
    """Reverse sweep over the tape of diff_forward. Returns (grad4, g_pveg, g_pden)
    for grad4 = dL/d(p_h, c1, c2, a)."""
    H, W = S0.shape
    burn = (np.asarray(S0) != 0).astype(np.uint8)
    T = len(tape)
    la, lb = _f64(la_T).copy(), _f64(lb_T).copy()
    g4 = np.zeros(4)
    gpv = np.zeros((H, W))
    gpd = np.zeros((H, W))
    cur_e, q, Gq = None, None, None

    def flush(e):
        V, th = winds[e]
        g, pv, pd = prep_adjoint(H, W, land.E, land.p_veg, land.p_den, V, th, prm, Gq, burnable=burn)
        return g, pv, pd

    for t in range(T - 1, -1, -1):
        e = _epoch_of(t, starts)
        if e != cur_e:
            if cur_e is not None:
                g, pv, pd = flush(cur_e)
                g4 += g; gpv += pv; gpd += pd
            cur_e = e
            V, th = winds[e]
            q = prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=burn)
            Gq = np.zeros((8, H, W))
        a, b = tape[t]
        la, lb = adjoint_step(a, b, q, prm.p_continue, la, lb, Gq)
    if cur_e is not None:
        g, pv, pd = flush(cur_e)
        g4 += g; gpv += pv; gpd += pd
    return g4, gpv, gpd


# --------------------------------------------------------------------- loss

BCE_EPS = 1e-7


def bce(a_T, y):
    """Mean binary cross-entropy of yhat = clamp(a_T, eps, 1-eps) against y in {0,1};
    returns (loss, dL/da_T). The clamp passes no gradient outside [eps, 1-eps]."""
    a_T = _f64(a_T)
    y = _f64(y)
    N = a_T.size
    yh = np.clip(a_T, BCE_EPS, 1.0 - BCE_EPS)
    loss = -np.mean(y * np.log(yh) + (1.0 - y) * np.log(1.0 - yh))
    inside = (a_T >= BCE_EPS) & (a_T <= 1.0 - BCE_EPS)
    g = np.where(inside, (yh - y) / (yh * (1.0 - yh)) / N, 0.0)
    return float(loss), g
