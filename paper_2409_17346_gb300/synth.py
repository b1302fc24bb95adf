"""Seeded synthetic inputs shaped like the paper's workloads.

This module only generates data: original fields f, emulated base-compressor outputs
f_hat, and the absolute error bound xi.  It holds none of the method's arithmetic and is
the only code shared by the CUDA path's tests/benchmarks and the CPU oracle's tests.

Fields are float32 numpy arrays of shape (ny, nx) in 2D or (nz, ny, nx) in 3D (x fastest).
The paper's datasets and base compressors (SZ3, ZFP, SPERR, MGARD) are not available;
these recipes stand in for them:

* ``gaussians_2d``  -- sum of 8 Gaussian bumps plus small white noise (a 64x64 case).
* ``multiscale_2d`` -- 64 random-phase plane waves plus 4-octave value noise, a smooth
  climate-like field (stands in for CESM 3600x1800).
* ``grf_3d``        -- isotropic Gaussian random field, power spectrum P(k) ~ k^slope,
  by seeded FFT synthesis (slope -3 for the 256^3 case; slope -11/3 gives the
  Kolmogorov k^-5/3 shell spectrum for the 512^3 turbulence-like case).
* ``add_plateaus``  -- replaces a cube covering ~5% of the volume by 16^3 tiles of
  constant value (each tile's float32 mean) to exercise index tie-breaking.
* ``noise_base`` / ``quantize_dither_base`` -- base-compressor emulators: uniform noise
  in [-xi, xi], or uniform quantisation to bins of width 2 xi plus a +-xi dither.
"""
import math

import numpy as np

__all__ = ["xi_from_range", "gaussians_2d", "multiscale_2d", "grf_3d", "add_plateaus",
           "noise_base", "quantize_dither_base", "config_case", "serving_requests", "extreme_noise_2d"]


def xi_from_range(f, rel):
    """xi = fl32(rel * fl32(max - min))."""
    rng = np.float32(np.float32(f.max()) - np.float32(f.min()))
    return float(np.float32(np.float32(rel) * rng))


def gaussians_2d(nx=64, ny=64, seed=1, n_bumps=8, noise_std=1e-3):
    r = np.random.Generator(np.random.PCG64(seed))
    cx = r.uniform(0, nx, n_bumps)
    cy = r.uniform(0, ny, n_bumps)
    sig = r.uniform(3.0, 10.0, n_bumps)
    amp = r.uniform(-1.0, 1.0, n_bumps)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    f = np.zeros((ny, nx))
    for i in range(n_bumps):
        f += amp[i] * np.exp(-((x - cx[i]) ** 2 + (y - cy[i]) ** 2) / (2 * sig[i] ** 2))
    f += r.normal(0.0, noise_std, (ny, nx))
    return f.astype(np.float32)


def _value_noise(r, nx, ny, lattice):
    gx = nx // lattice + 2
    gy = ny // lattice + 2
    vals = r.uniform(-1.0, 1.0, (gy, gx))
    xs = np.arange(nx) / lattice
    ys = np.arange(ny) / lattice
    x0 = np.floor(xs).astype(np.int64)
    y0 = np.floor(ys).astype(np.int64)
    tx = xs - x0
    ty = ys - y0
    sx = tx * tx * (3 - 2 * tx)
    sy = ty * ty * (3 - 2 * ty)
    v00 = vals[y0][:, x0]
    v01 = vals[y0][:, x0 + 1]
    v10 = vals[y0 + 1][:, x0]
    v11 = vals[y0 + 1][:, x0 + 1]
    top = v00 + (v01 - v00) * sx[None, :]
    bot = v10 + (v11 - v10) * sx[None, :]
    return top + (bot - top) * sy[:, None]


def multiscale_2d(nx=3600, ny=1800, seed=2, n_waves=64, lam_min=20.0, lam_max=900.0,
                  noise_rel=0.05):
    r = np.random.Generator(np.random.PCG64(seed))
    theta = r.uniform(0.0, math.pi, n_waves)
    lam = np.exp(r.uniform(math.log(lam_min), math.log(lam_max), n_waves))
    phase = r.uniform(0.0, 2 * math.pi, n_waves)
    amp = lam / lam_max
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    kx = 2 * np.pi * np.cos(theta) / lam
    ky = 2 * np.pi * np.sin(theta) / lam
    ax = np.outer(kx, xs) + phase[:, None]          # (waves, nx)
    ay = np.outer(ys, ky)                           # (ny, waves)
    # sum_i amp_i sin(ax_i + ay_i), with sin(a + b) = sin a cos b + cos a sin b: two products
    f = (np.cos(ay) * amp) @ np.sin(ax) + (np.sin(ay) * amp) @ np.cos(ax)
    noise = np.zeros((ny, nx))
    gain = 1.0
    for lattice in (64, 32, 16, 8):
        noise += gain * _value_noise(r, nx, ny, lattice)
        gain *= 0.5
    noise *= noise_rel * f.std() / max(noise.std(), 1e-30)
    return (f + noise).astype(np.float32)


def grf_3d(n=64, seed=3, slope=-3.0, shape=None):
    """Gaussian random field with P(k) ~ |k|^slope, P(0) = 0, normalised to [0, 1]."""
    import torch
    nz, ny, nx = shape if shape is not None else (n, n, n)
    r = np.random.Generator(np.random.PCG64(seed))
    white = torch.from_numpy(r.standard_normal((nz, ny, nx), dtype=np.float32))
    spec = torch.fft.rfftn(white)
    kz = torch.fft.fftfreq(nz).reshape(-1, 1, 1)
    ky = torch.fft.fftfreq(ny).reshape(1, -1, 1)
    kx = torch.fft.rfftfreq(nx).reshape(1, 1, -1)
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2.pow(slope / 4.0)          # sqrt(P) = |k|^(slope/2)
    amp[0, 0, 0] = 0.0
    spec *= amp
    del amp, k2
    f = torch.fft.irfftn(spec, s=(nz, ny, nx))
    del spec
    lo, hi = f.min(), f.max()
    f = (f - lo) / (hi - lo)
    return f.numpy().astype(np.float32)


def add_plateaus(f, seed, frac=0.05, tile=16):
    """Overwrite a seeded cube (side ceil(frac^(1/3) * n)) with tile^3 blocks, each set to
    its own float32 mean, so that large groups of vertices tie exactly."""
    f = f.copy()
    nz, ny, nx = f.shape
    side = int(math.ceil(frac ** (1.0 / 3.0) * min(nx, ny, nz)))
    r = np.random.Generator(np.random.PCG64(seed + 7919))
    oz = int(r.integers(0, nz - side + 1))
    oy = int(r.integers(0, ny - side + 1))
    ox = int(r.integers(0, nx - side + 1))
    for z in range(oz, oz + side, tile):
        for y in range(oy, oy + side, tile):
            for x in range(ox, ox + side, tile):
                z1, y1, x1 = min(z + tile, oz + side), min(y + tile, oy + side), min(x + tile, ox + side)
                blk = f[z:z1, y:y1, x:x1]
                blk[...] = np.float32(blk.astype(np.float64).mean())
    return f


def noise_base(f, xi, seed):
    """Emulated base compressor: f + U[-xi, xi] (float32)."""
    r = np.random.Generator(np.random.PCG64(seed + 104729))
    d = r.uniform(-xi, xi, f.shape).astype(np.float32)
    return (f + d).astype(np.float32)


def quantize_dither_base(f, xi, seed):
    """Emulated base compressor: bins of width 2 xi plus a +-xi dither (may exceed xi)."""
    r = np.random.Generator(np.random.PCG64(seed + 104729))
    q = np.round(f.astype(np.float64) / (2 * xi)) * (2 * xi)
    d = r.uniform(-xi, xi, f.shape)
    return (q + d).astype(np.float32)


def config_case(name, seed=None, rel=None, size=None):
    """(f, f_hat, xi, tier) for one of the named workloads.

    name: 'gauss2d' (64x64, T3), 'multiscale2d' (1800x3600, T4), 'grf3d' (256^3, T4),
    'kolmogorov3d' (512^3 with plateaus, T4).  ``size`` shrinks a case for tests
    (an int side for 3D, an (ny, nx) pair for 2D)."""
    if name == "gauss2d":
        seed = 1 if seed is None else seed
        ny, nx = size if size is not None else (64, 64)
        f = gaussians_2d(nx, ny, seed)
        xi = xi_from_range(f, 1e-3 if rel is None else rel)
        return f, noise_base(f, xi, seed), xi, 3
    if name == "multiscale2d":
        seed = 2 if seed is None else seed
        ny, nx = size if size is not None else (1800, 3600)
        f = multiscale_2d(nx, ny, seed)
        xi = xi_from_range(f, 1e-3 if rel is None else rel)
        return f, quantize_dither_base(f, xi, seed), xi, 4
    if name == "grf3d":
        seed = 3 if seed is None else seed
        n = size if size is not None else 256
        f = grf_3d(n, seed, -3.0)
        xi = xi_from_range(f, 1e-4 if rel is None else rel)
        return f, noise_base(f, xi, seed), xi, 4
    if name == "kolmogorov3d":
        seed = 4 if seed is None else seed
        n = size if size is not None else 512
        f = add_plateaus(grf_3d(n, seed, -11.0 / 3.0), seed)
        xi = xi_from_range(f, 1e-4 if rel is None else rel)
        return f, noise_base(f, xi, seed), xi, 4
    raise ValueError(name)


def extreme_noise_2d(n, seed=9, xi=1e-4):
    """The stress case of the paper's extreme-case study: an n x n field of white noise whose
    whole range lies inside the error bound (values U[0, xi]), and a base-compressor output
    that is flat (every value xi / 2), so that the local order is destroyed everywhere.
    Returns (f, f_hat, xi); f_hat lies within xi of f at every vertex."""
    r = np.random.Generator(np.random.PCG64(seed))
    xi32 = np.float32(xi)
    f = r.uniform(0.0, float(xi32), (n, n)).astype(np.float32)
    fh = np.full_like(f, np.float32(xi32 / np.float32(2)))
    return f, fh, float(xi32)


def serving_requests(n=128, seed=5, rate_hz=20.0):
    """Arrival schedule for the serving workload: list of dicts with arrival time (s),
    kind ('2d' side or '3d' side), seed and relative bound."""
    r = np.random.Generator(np.random.PCG64(seed))
    gaps = r.exponential(1.0 / rate_hz, n)
    t = np.cumsum(gaps) - gaps[0]
    sizes = [("2d", 256), ("2d", 1024), ("2d", 2048), ("3d", 64), ("3d", 128), ("3d", 256)]
    out = []
    for i in range(n):
        kind, side = sizes[int(r.integers(0, len(sizes)))]
        rel = (1e-3, 1e-4)[int(r.integers(0, 2))]
        out.append(dict(t=float(t[i]), kind=kind, side=side, seed=1000 + i, rel=rel))
    return out


def serving_field(req):
    """(f, f_hat, xi) for one serving request: config-2-like 2D or config-3-like 3D."""
    if req["kind"] == "2d":
        s = req["side"]
        f = multiscale_2d(s, s, req["seed"])
        xi = xi_from_range(f, req["rel"])
        return f, quantize_dither_base(f, xi, req["seed"]), xi
    s = req["side"]
    f = grf_3d(s, req["seed"], -3.0)
    xi = xi_from_range(f, req["rel"])
    return f, noise_base(f, xi, req["seed"]), xi
