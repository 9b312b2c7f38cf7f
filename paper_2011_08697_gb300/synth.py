"""Seeded synthetic scalar fields for critical-point tracking.

This module only *samples* fields; it holds none of the tracking method's
arithmetic (no quantisation, no gradients, no predicates).  It is the single
piece of code shared by the CUDA path's tests/bench and the CPU oracle, so
that both sides always see the same float32 array.

Layout of every field: C-contiguous float32, ``f[t][y][x]`` in 2D and
``f[t][z][y][x]`` in 3D (x fastest).

Workloads (shapes follow the paper's synthetic and application data):

* spiral woven (Sec. 4.4, "2D spiral woven with perturbations"):
  f = cos(x cos t - y sin t) * sin(x sin t + y cos t) on an inclusive
  linspace grid over [-4, 4]^2, t_k = k/(nt-1) over [0, 1], optional i.i.d.
  Gaussian noise added in FP64 before a single cast to float32.
* moving minimum (Sec. 4.4, "3D moving minimum"):
  f = |x - (x0 + d t)|^2 on an integer grid, t = step index; with dyadic d
  every sample is exact in float32.
* moving Gaussian blobs: a seeded sum of Gaussians moving on linear paths,
  standing in for the 128^3 turbulent-vortex data of Sec. 4.5 (the dataset
  itself is not available).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "spiral_woven",
    "moving_minimum",
    "gaussian_blobs",
    "random_levels",
    "BlobSet",
    "blob_set",
    "blob_slice",
    "batch_fields",
    "stream_specs",
    "poisson_arrivals",
    "linear_vector_field",
    "vortex_street",
]


def spiral_woven(n: int, nt: int, sigma: float = 0.0, seed: int = 0,
                 lo: float = -4.0, hi: float = 4.0, ny: int | None = None,
                 k_stop: int | None = None) -> np.ndarray:
    """Spiral woven field sampled on an ``ny x n`` grid over ``nt`` steps.

    x_i = lo + (hi-lo) i/(n-1) (inclusive linspace), t_k = k/(nt-1).
    Noise N(0, sigma^2) is drawn slice by slice from ``default_rng(seed)``.
    ``k_stop`` returns only the first k_stop slices (identical to the leading
    slices of the full field).
    """
    ny = n if ny is None else ny
    x = np.linspace(lo, hi, n)
    y = np.linspace(lo, hi, ny)
    ts = np.linspace(0.0, 1.0, nt) if nt > 1 else np.zeros(1)
    rng = np.random.default_rng(seed)
    if k_stop is not None:
        ts = ts[:k_stop]
    out = np.empty((len(ts), ny, n), dtype=np.float32)
    X = x[None, :]
    Y = y[:, None]
    for k, t in enumerate(ts):
        c, s = math.cos(t), math.sin(t)
        f = np.cos(X * c - Y * s) * np.sin(X * s + Y * c)
        if sigma > 0.0:
            f = f + sigma * rng.standard_normal((ny, n))
        out[k] = f
    return out


def moving_minimum(n: int, nt: int, x0, d, ndim: int = 3) -> np.ndarray:
    """f(x, t) = |x - (x0 + d t)|^2 on the integer grid {0..n-1}^ndim, t = 0..nt-1.

    With x0 and d dyadic (e.g. multiples of 1/4) every value is exact in
    float32, so the minimum's trajectory x0 + d t is known exactly.
    """
    x0 = np.asarray(x0, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    assert x0.shape == (ndim,) and d.shape == (ndim,)
    idx = np.arange(n, dtype=np.float64)
    shape = (nt,) + (n,) * ndim
    out = np.empty(shape, dtype=np.float32)
    for k in range(nt):
        c = x0 + d * k
        f = np.zeros((n,) * ndim, dtype=np.float64)
        for a in range(ndim):
            # axis a of the point maps to array axis (ndim-1-a): x is fastest
            sh = [1] * ndim
            sh[ndim - 1 - a] = n
            f = f + ((idx - c[a]) ** 2).reshape(sh)
        out[k] = f
    return out


def random_levels(shape, levels=(-1.0, 0.0, 1.0), seed: int = 0) -> np.ndarray:
    """A field whose samples are drawn uniformly from a few levels.

    With levels {-1, 0, 1} almost every simplex is degenerate, which is the
    hardest case for the symbolic perturbation.
    """
    rng = np.random.default_rng(seed)
    lv = np.asarray(levels, dtype=np.float32)
    return lv[rng.integers(0, len(lv), size=shape)].astype(np.float32)


@dataclass
class BlobSet:
    """Parameters of a sum of moving Gaussians (grid-index units)."""
    centre: np.ndarray     # (nb, ndim) at t=0, axis order x, y, (z)
    sigma: np.ndarray      # (nb,)
    amp: np.ndarray        # (nb,)
    vel: np.ndarray        # (nb, ndim) cells per step
    dims: tuple            # (nx, ny[, nz])


def blob_set(dims, nblobs: int, seed: int, sigma_range=(4.0, 12.0),
             amp_range=(0.5, 1.0), vmax: float = 1.0) -> BlobSet:
    """Draw centres U[0,N) per axis, sigma U[sigma_range], amplitude
    +-U[amp_range] with a random sign, velocity = uniform random direction
    times U[0, vmax] cells/step."""
    rng = np.random.default_rng(seed)
    ndim = len(dims)
    centre = rng.uniform(0.0, 1.0, size=(nblobs, ndim)) * np.asarray(dims, dtype=np.float64)
    sigma = rng.uniform(sigma_range[0], sigma_range[1], size=nblobs)
    amp = rng.uniform(amp_range[0], amp_range[1], size=nblobs)
    amp = amp * np.where(rng.integers(0, 2, size=nblobs) == 0, -1.0, 1.0)
    direc = rng.standard_normal((nblobs, ndim))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    speed = rng.uniform(0.0, vmax, size=nblobs)
    vel = direc * speed[:, None]
    return BlobSet(centre, sigma, amp, vel, tuple(int(v) for v in dims))


def blob_slice(bs: BlobSet, k: int) -> np.ndarray:
    """One time slice (float32, z/y/x order) of a moving blob field at step k."""
    dims = bs.dims
    ndim = len(dims)
    out = np.zeros(tuple(reversed(dims)), dtype=np.float64)
    for b in range(len(bs.sigma)):
        c = bs.centre[b] + bs.vel[b] * k
        inv = 1.0 / (2.0 * bs.sigma[b] ** 2)
        term = None
        for a in range(ndim):
            coord = np.arange(dims[a], dtype=np.float64)
            e = np.exp(-((coord - c[a]) ** 2) * inv)
            sh = [1] * ndim
            sh[ndim - 1 - a] = dims[a]
            e = e.reshape(sh)
            term = e if term is None else term * e
        out += bs.amp[b] * term
    return out.astype(np.float32)


def gaussian_blobs(dims, nt: int, nblobs: int = 32, seed: int = 0, **kw) -> np.ndarray:
    """A full (nt, [nz,] ny, nx) float32 field of moving Gaussian blobs."""
    bs = blob_set(dims, nblobs, seed, **kw)
    out = np.empty((nt,) + tuple(reversed(dims)), dtype=np.float32)
    for k in range(nt):
        out[k] = blob_slice(bs, k)
    return out


def batch_fields(count: int = 256, n_lo: int = 64, n_hi: int = 512, nt_lo: int = 8,
                 nt_hi: int = 32, nb_lo: int = 8, nb_hi: int = 64, seed0: int = 0,
                 materialise: bool = True):
    """Many independent 2D blob fields of uneven size and length.

    Field i uses seed ``seed0 + i``: N = round(exp(U[ln n_lo, ln n_hi])) for a
    square N x N grid, nt ~ U{nt_lo..nt_hi}, nblobs ~ U{nb_lo..nb_hi}, sigma
    scaled by N/128.  Returns a list of (nx, ny, nt, array-or-None, BlobSet).
    """
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        nt = int(rng.integers(nt_lo, nt_hi + 1))
        nb = int(rng.integers(nb_lo, nb_hi + 1))
        scale = n / 128.0
        bs = blob_set((n, n), nb, seed=10_000 + seed0 + i,
                      sigma_range=(4.0 * scale, 12.0 * scale), vmax=1.0)
        arr = None
        if materialise:
            arr = np.empty((nt, n, n), dtype=np.float32)
            for k in range(nt):
                arr[k] = blob_slice(bs, k)
        out.append((n, n, nt, arr, bs))
    return out


def stream_specs(count: int = 32, n_lo: int = 256, n_hi: int = 2048, seed0: int = 0,
                 nb_lo: int = 8, nb_hi: int = 64):
    """Per-stream grid size (log-uniform square N) and blob parameters."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(50_000 + seed0 + i)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        nb = int(rng.integers(nb_lo, nb_hi + 1))
        scale = n / 128.0
        bs = blob_set((n, n), nb, seed=60_000 + seed0 + i,
                      sigma_range=(4.0 * scale, 12.0 * scale), vmax=1.0)
        out.append((n, bs))
    return out


def poisson_arrivals(nstreams: int, rate_total: float, duration_s: float, seed: int = 0):
    """Merged Poisson arrival process: list of (time_s, stream_index), sorted.

    Each stream gets an independent Poisson process of rate rate_total/nstreams.
    """
    rng = np.random.default_rng(seed)
    lam = rate_total / nstreams
    events = []
    for s in range(nstreams):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / lam)
            if t > duration_s:
                break
            events.append((t, s))
    events.sort()
    return events


def blob_slices_torch(bs: BlobSet, k0: int, k1: int, device, chunk: int = 16):
    """Slices k0..k1-1 of a 2D moving blob field as one float32 torch tensor
    (k1-k0, ny, nx) computed on ``device``: the law of :func:`blob_slice`
    (sum over blobs of separable Gaussians, FP64, cast once to float32),
    written as a product over the blob axis.  Values may differ from the NumPy
    generator in the last bit; both tracking sides always read the same
    float32 array."""
    import torch
    nx, ny = bs.dims
    f64 = torch.float64
    cx = torch.as_tensor(bs.centre[:, 0], dtype=f64, device=device)
    cy = torch.as_tensor(bs.centre[:, 1], dtype=f64, device=device)
    vx = torch.as_tensor(bs.vel[:, 0], dtype=f64, device=device)
    vy = torch.as_tensor(bs.vel[:, 1], dtype=f64, device=device)
    inv = torch.as_tensor(1.0 / (2.0 * bs.sigma ** 2), dtype=f64, device=device)
    amp = torch.as_tensor(bs.amp, dtype=f64, device=device)
    xs = torch.arange(nx, dtype=f64, device=device)
    ys = torch.arange(ny, dtype=f64, device=device)
    out = torch.empty((k1 - k0, ny, nx), dtype=torch.float32, device=device)
    for a in range(k0, k1, chunk):
        ks = torch.arange(a, min(k1, a + chunk), dtype=f64, device=device)
        ccx = cx[None, :] + vx[None, :] * ks[:, None]            # (K, nb)
        ccy = cy[None, :] + vy[None, :] * ks[:, None]
        ex = torch.exp(-((xs[None, None, :] - ccx[:, :, None]) ** 2) * inv[None, :, None])   # (K, nb, nx)
        ey = torch.exp(-((ys[None, None, :] - ccy[:, :, None]) ** 2) * inv[None, :, None])   # (K, nb, ny)
        ey = ey * amp[None, :, None]
        out[a - k0: a - k0 + len(ks)] = torch.bmm(ey.transpose(1, 2), ex).to(torch.float32)
    return out


def linear_vector_field(n: int, nt: int, A, c0, d) -> np.ndarray:
    """v(x, t) = A (x - c0 - d t) on the integer grid {0..n-1}^2, t = 0..nt-1,
    as a (nt, n, n, 2) float32 array (component 0 = x).  With dyadic A, c0
    and d every value is exact in float32; the only zero at time t is
    c0 + d t when A is regular."""
    A = np.asarray(A, dtype=np.float64)
    c0 = np.asarray(c0, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    idx = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(idx, idx)            # [y][x]
    out = np.empty((nt, n, n, 2), dtype=np.float32)
    for k in range(nt):
        cx, cy = c0 + d * k
        dx, dy = X - cx, Y - cy
        out[k, :, :, 0] = A[0, 0] * dx + A[0, 1] * dy
        out[k, :, :, 1] = A[1, 0] * dx + A[1, 1] * dy
    return out


def vortex_street(nx: int, ny: int, nt: int, nvort: int = 8, nsrc: int = 6, seed: int = 0,
                  flow: float = 0.3, sigma=(3.0, 6.0), drift: float = 0.5) -> np.ndarray:
    """A 2D vector field shaped like the wake behind a cylinder (a stand-in
    for the flow-past-cylinder data, which is not available): a uniform flow
    along x plus a double row of Gaussian vortices of alternating sign,
    advected downstream by `drift` cells per step, plus a few Gaussian
    sources and sinks (gradients of Gaussian bumps) so that every kind of
    zero occurs.  (nt, ny, nx, 2) float32, component 0 = x, values in FP64
    cast once."""
    rng = np.random.default_rng(seed)
    xs = np.arange(nx, dtype=np.float64)[None, :]
    ys = np.arange(ny, dtype=np.float64)[:, None]
    x0 = rng.uniform(0.0, nx, size=nvort)
    y0 = ny / 2.0 + np.where(np.arange(nvort) % 2 == 0, 1.0, -1.0) * rng.uniform(ny / 8.0, ny / 4.0, size=nvort)
    gam = np.where(np.arange(nvort) % 2 == 0, 1.0, -1.0) * rng.uniform(0.5, 1.0, size=nvort)
    sv = rng.uniform(sigma[0], sigma[1], size=nvort)
    sx = rng.uniform(0.0, nx, size=nsrc)
    sy = rng.uniform(0.0, ny, size=nsrc)
    sa = np.where(rng.integers(0, 2, size=nsrc) == 0, -1.0, 1.0) * rng.uniform(0.5, 1.0, size=nsrc)
    ss = rng.uniform(sigma[0], sigma[1], size=nsrc)
    out = np.empty((nt, ny, nx, 2), dtype=np.float32)
    for k in range(nt):
        u = np.full((ny, nx), flow)
        w = np.zeros((ny, nx))
        for i in range(nvort):
            dx = xs - (x0[i] + drift * k)
            dy = ys - y0[i]
            g = np.exp(-(dx * dx + dy * dy) / (2.0 * sv[i] ** 2)) / sv[i]
            u += -gam[i] * dy * g / sv[i]
            w += gam[i] * dx * g / sv[i]
        for j in range(nsrc):
            dx = xs - sx[j]
            dy = ys - sy[j]
            g = np.exp(-(dx * dx + dy * dy) / (2.0 * ss[j] ** 2))
            u += -sa[j] * dx * g / ss[j]
            w += -sa[j] * dy * g / ss[j]
        out[k, :, :, 0] = u
        out[k, :, :, 1] = w
    return out
