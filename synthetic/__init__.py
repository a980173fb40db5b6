"""Seeded synthetic landscapes and ignitions for the wildfire cellular automaton.

This module is shared by the tests, the benchmark and the CPU oracle as a source of
*inputs only*. It contains none of the automaton's arithmetic: no propagation
probability, no slope or wind factor, no ignition rule. Every array it returns is a
plain float32 (fields) or uint8 (states) numpy array in row-major H x W layout.

Recipe (stated once here, used everywhere):

* Elevation E: white N(0,1) noise, Gaussian-filtered with sigma = 8 cells in Fourier
  space (periodic), scaled to E = 200 m * g / max|g|.
* Vegetation p_veg: uniform choice from {-0.3, 0, 0.4}; density p_den: uniform choice
  from {-0.4, 0, 0.3}.
* Non-burnable cells: Bernoulli(0.05), written as state 0 of the initial state.
* Wind: either uniform (V_w, theta_w) or smooth random fields with correlation length
  about 32 cells: V_w = 12 m/s * (g - min)/(max - min), theta_w = 360 deg * (g' - min)/(max - min).
  Smooth fields with sigma >= 16 are drawn on a grid 8x coarser (sigma/8 there) and
  bilinearly upsampled, which keeps 8192^2 wind epochs cheap to generate.
* Ignitions: the centre cell, or 1-5 random burnable cells.

All draws come from numpy ``Generator(PCG64(seed))`` streams; float64 draws are cast to
float32 at the end. The paper's real landscapes (LANDFIRE, ERA5, MODIS) are not
available; these fields stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "smooth_field",
    "Landscape",
    "make_landscape",
    "uniform_wind",
    "smooth_wind",
    "initial_state",
    "random_state",
    "CONFIG1",
]


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _gauss_filter_fft(x: np.ndarray, sigma: float) -> np.ndarray:
    ky = np.fft.fftfreq(x.shape[0])[:, None]
    kx = np.fft.rfftfreq(x.shape[1])[None, :]
    g = np.exp(-2.0 * math.pi ** 2 * sigma * sigma * (ky * ky + kx * kx))
    try:
        import scipy.fft as sf

        X = sf.rfft2(x, workers=-1)
        return sf.irfft2(X * g, s=x.shape, workers=-1)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        return np.fft.irfft2(np.fft.rfft2(x) * g, s=x.shape)


def _bilinear_upsample(x: np.ndarray, H: int, W: int, f: int) -> np.ndarray:
    """Upsample a coarse periodic field by integer factor f (cell-centred, wraps);
    separable: along columns on the coarse rows first, then along rows. Uses torch's
    multi-threaded CPU ops when available (same arithmetic as the numpy fallback)."""
    h, w = x.shape
    ry = (np.arange(H) + 0.5) / f - 0.5
    rx = (np.arange(W) + 0.5) / f - 0.5
    y0 = np.floor(ry).astype(np.int64)
    x0 = np.floor(rx).astype(np.int64)
    fy = (ry - y0).astype(np.float32)[:, None]
    fx = (rx - x0).astype(np.float32)[None, :]
    try:
        import torch
        xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
        cols = torch.lerp(xt[:, torch.from_numpy(x0 % w)], xt[:, torch.from_numpy((x0 + 1) % w)],
                          torch.from_numpy(fx))
        out = torch.lerp(cols[torch.from_numpy(y0 % h)], cols[torch.from_numpy((y0 + 1) % h)],
                         torch.from_numpy(fy))
        return out.numpy()
    except ImportError:  # pragma: no cover
        cols = x[:, x0 % w] * (1 - fx) + x[:, (x0 + 1) % w] * fx          # h x W
        return cols[y0 % h] * (1 - fy) + cols[(y0 + 1) % h] * fy           # H x W


def smooth_field(H: int, W: int, sigma: float, seed: int, stream: int = 0) -> np.ndarray:
    """Zero-mean smooth random field (float32, H x W) with correlation length ~sigma cells."""
    rng = _rng(seed, stream)
    if sigma >= 16:
        f = 8
        h, w = -(-H // f), -(-W // f)
        noise = rng.standard_normal((h, w))
        g = _gauss_filter_fft(noise, sigma / f)
        g = _bilinear_upsample(g.astype(np.float32), H, W, f)
    else:
        # FP64 noise and transform: their FP32 rounding comes out the same on x86 and Arm
        # hosts (an FP32 transform does not), so both build identical fields
        noise = rng.standard_normal((H, W))
        g = _gauss_filter_fft(noise, sigma)
    return np.ascontiguousarray(g, dtype=np.float32)


@dataclasses.dataclass
class Landscape:
    """Static per-cell fields (float32, H x W, row-major) and the non-burnable mask."""

    E: np.ndarray
    p_veg: np.ndarray
    p_den: np.ndarray
    burnable: np.ndarray  # uint8, 1 burnable / 0 non-burnable

    @property
    def shape(self):
        return self.E.shape


def make_landscape(H: int, W: int, seed: int, nonburnable_frac: float = 0.05,
                   sigma_E: float = 8.0, amp_E: float = 200.0) -> Landscape:
    g = smooth_field(H, W, sigma_E, seed, stream=1).astype(np.float64)
    m = np.max(np.abs(g))
    E = (amp_E * g / m) if m > 0 else np.zeros_like(g)
    rng = _rng(seed, 2)
    p_veg = rng.choice(np.array([-0.3, 0.0, 0.4]), size=(H, W))
    p_den = rng.choice(np.array([-0.4, 0.0, 0.3]), size=(H, W))
    burnable = (rng.random((H, W)) >= nonburnable_frac).astype(np.uint8)
    return Landscape(E=E.astype(np.float32), p_veg=p_veg.astype(np.float32),
                     p_den=p_den.astype(np.float32), burnable=burnable)


def uniform_wind(H: int, W: int, V: float, theta_deg: float):
    return (np.full((H, W), V, dtype=np.float32), np.full((H, W), theta_deg, dtype=np.float32))


def _rescale(g: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """lo + (hi - lo) (g - min)/(max - min), computed in float32."""
    g = np.asarray(g, dtype=np.float32)
    mn, mx = float(g.min()), float(g.max())
    if mx <= mn:
        return np.full(g.shape, lo, dtype=np.float32)
    out = g - np.float32(mn)
    out *= np.float32((hi - lo) / (mx - mn))
    out += np.float32(lo)
    return out


def smooth_wind(H: int, W: int, seed: int, epoch: int = 0, sigma: float = 32.0,
                v_max: float = 12.0):
    """Smooth random wind epoch: (V_w in [0, v_max] m/s, theta_w in [0, 360] degrees)."""
    gv = smooth_field(H, W, sigma, seed + epoch, stream=3)
    gt = smooth_field(H, W, sigma, seed + epoch, stream=4)
    return _rescale(gv, 0.0, v_max), _rescale(gt, 0.0, 360.0)


def initial_state(land: Landscape, ignitions) -> np.ndarray:
    """uint8 H x W state: 0 non-burnable, 1 unburned, 2 burning at the ignition cells."""
    S = np.where(land.burnable != 0, 1, 0).astype(np.uint8)
    for (r, c) in ignitions:
        S[r, c] = 2
    return S


def random_ignitions(land: Landscape, seed: int, n_min: int = 1, n_max: int = 5):
    rng = _rng(seed, 5)
    n = int(rng.integers(n_min, n_max + 1))
    cand = np.argwhere(land.burnable != 0)
    idx = rng.choice(len(cand), size=min(n, len(cand)), replace=False)
    return [tuple(int(v) for v in cand[i]) for i in idx]


def random_state(H: int, W: int, seed: int, probs=(0.05, 0.55, 0.25, 0.15), R: int | None = None) -> np.ndarray:
    """Random (not fire-shaped) uint8 states in {0,1,2,3} for single-step parity tests."""
    rng = _rng(seed, 6)
    shape = (H, W) if R is None else (R, H, W)
    return rng.choice(np.arange(4, dtype=np.uint8), size=shape, p=np.asarray(probs))


def random_diff_state(H: int, W: int, seed: int, burnable: np.ndarray | None = None):
    """Random continuous state (a, b) with 0 <= b <= a <= 1, zero where not burnable."""
    rng = _rng(seed, 7)
    a = rng.random((H, W))
    b = a * rng.random((H, W))
    # sprinkle exact 0/1 values: the kernels must handle the saturated corners
    z = rng.random((H, W))
    a = np.where(z < 0.1, 0.0, a)
    b = np.where(z < 0.1, 0.0, b)
    a = np.where(z > 0.95, 1.0, a)
    b = np.where(z > 0.97, 1.0, np.where(z > 0.95, 0.0, b))
    if burnable is not None:
        a = np.where(burnable != 0, a, 0.0)
        b = np.where(burnable != 0, b, 0.0)
    return a.astype(np.float32), b.astype(np.float32)


# The small plain-forward workload: 128 x 128, l = 30 m, T = 200, uniform wind 5 m/s at
# 45 degrees, parameters below, one ignited centre cell, Philox seed 0, fields seed 0.
CONFIG1 = dict(H=128, W=128, T=200, l=30.0, V=5.0, theta=45.0, p_h=0.58, c1=0.045,
               c2=0.131, a=0.078, p_continue=0.3, seed=0, field_seed=0)
