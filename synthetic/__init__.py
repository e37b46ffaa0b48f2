"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the oracle tests, the CUDA parity tests and the
benchmark.  It holds no arithmetic of the MPR method itself (no angle map,
no energy, no Monte Carlo step): it only draws gridded fields and gap masks.

* Gaussian random fields with Whittle-Matern covariance (Sec. 4.1, eq. of the
  WM covariance), sampled with the circulant-embedding FFT method (Dietrich &
  Newsam 1997; Wood & Chan 1994).  The inverse autocorrelation length is
  kappa = 1/ell.
* Non-Gaussian marginals: lognormal (Sec. 4.3, log Z normal) and a gamma
  marginal obtained by a Gaussian-copula transform.
* Missing-data patterns of Sec. 4.1: removal of exactly floor(p * N_G) random
  points, and solid rectangular blocks.

Every function is deterministic given its integer seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.fft
import scipy.special
import scipy.stats

__all__ = [
    "matern_cov", "grf", "lognormal_grf", "gamma_grf", "uniform_gaps",
    "block_gaps", "Workload", "workload", "WORKLOADS",
]


def matern_cov(h, sigma: float, nu: float, ell: float):
    """Whittle-Matern covariance 2^(1-nu) sigma^2 / Gamma(nu) (k h)^nu K_nu(k h), k = 1/ell."""
    h = np.asarray(h, dtype=np.float64)
    kh = h / ell
    if nu == 0.5:
        return sigma * sigma * np.exp(-kh)
    out = np.empty_like(kh)
    zero = kh == 0
    khn = kh[~zero]
    out[~zero] = (sigma * sigma * 2.0 ** (1.0 - nu) / scipy.special.gamma(nu)
                  * khn ** nu * scipy.special.kv(nu, khn))
    out[zero] = sigma * sigma
    return out


def grf(shape, *, nu: float, ell: float, mean: float = 0.0, std: float = 1.0,
        seed: int = 0, dtype=np.float64):
    """Stationary Gaussian random field on a (Ly, Lx) grid by circulant embedding.

    The covariance is embedded in a periodic torus of at least twice the grid
    size; negative eigenvalues of the embedding (a truncation artefact for
    long-range covariances) are clipped to zero.
    """
    Ly, Lx = int(shape[0]), int(shape[1])
    My = scipy.fft.next_fast_len(2 * Ly)
    Mx = scipy.fft.next_fast_len(2 * Lx)
    iy = np.arange(My)
    ix = np.arange(Mx)
    dy = np.minimum(iy, My - iy).astype(np.float64)
    dx = np.minimum(ix, Mx - ix).astype(np.float64)
    big = Lx * Ly > 1 << 22
    cdt = np.complex64 if big else np.complex128
    rdt = np.float32 if big else np.float64
    h = np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2)
    c = matern_cov(h, 1.0, nu, ell).astype(rdt)
    del h
    lam = scipy.fft.fft2(c, workers=-1).real
    del c
    np.maximum(lam, 0.0, out=lam)
    amp = np.sqrt(lam / (Mx * My)).astype(rdt)
    del lam
    rng = np.random.Generator(np.random.PCG64(seed))
    w = (rng.standard_normal((My, Mx), dtype=rdt)
         + 1j * rng.standard_normal((My, Mx), dtype=rdt)).astype(cdt)
    w *= amp
    del amp
    f = scipy.fft.fft2(w, workers=-1)
    y = np.ascontiguousarray(f.real[:Ly, :Lx]).astype(np.float64)
    return (mean + std * y).astype(dtype)


def lognormal_grf(shape, *, nu, ell, log_mean=0.0, log_std=1.0, seed=0):
    """Z = exp(Y) with Y a GRF of mean log_mean and std log_std."""
    return np.exp(grf(shape, nu=nu, ell=ell, mean=log_mean, std=log_std, seed=seed))


def gamma_grf(shape, *, nu, ell, k=2.0, theta=10.0, seed=0):
    """Gamma(shape k, scale theta) marginal through a Gaussian copula of a unit GRF."""
    y = grf(shape, nu=nu, ell=ell, seed=seed)
    u = scipy.special.ndtr(y)
    return scipy.stats.gamma.ppf(np.clip(u, 1e-15, 1 - 1e-15), a=k, scale=theta)


def uniform_gaps(shape, frac: float, seed: int):
    """Boolean mask (True = missing) with exactly floor(frac * N_G) random gaps (Sec. 4.1)."""
    n = int(shape[0]) * int(shape[1])
    p = int(math.floor(frac * n))
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.permutation(n)[:p]
    m = np.zeros(n, dtype=bool)
    m[idx] = True
    return m.reshape(shape)


def block_gaps(shape, rects):
    """Boolean mask with solid rectangles (y0, x0, h, w) removed (Sec. 4.1, case ii)."""
    m = np.zeros(shape, dtype=bool)
    for (y0, x0, h, w) in rects:
        m[y0:y0 + h, x0:x0 + w] = True
    return m


@dataclass
class Workload:
    """A set of images with their gap masks and the run parameters of one workload."""
    name: str
    z: list                      # per image float32 (Ly, Lx) with gap pixels holding the truth
    gap: list                    # per image uint8 (Ly, Lx), 1 = missing
    chains: int
    n_equil: int
    n_meas: int
    meta: dict = field(default_factory=dict)

    @property
    def shapes(self):
        return [g.shape for g in self.gap]

    @property
    def n_gap(self):
        return [int(g.sum()) for g in self.gap]


def _grf64(seed=1):
    z = grf((64, 64), nu=0.5, ell=8.0, mean=50.0, std=10.0, seed=seed)
    g = uniform_gaps((64, 64), 0.33, seed + 1)
    return Workload("grf64_p33", [z.astype(np.float32)], [g.astype(np.uint8)],
                    chains=10, n_equil=200, n_meas=100,
                    meta=dict(field="GRF N(50,10) exponential ell=8", gaps="33% uniform",
                              seed_field=seed, seed_mask=seed + 1))


def _lognormal1024(seed=11, L=1024):
    z = lognormal_grf((L, L), nu=1.5, ell=20.0, log_mean=0.0, log_std=0.8, seed=seed)
    g = uniform_gaps((L, L), 0.5, seed + 1)
    return Workload(f"lognormal{L}_p50", [z.astype(np.float32)], [g.astype(np.uint8)],
                    chains=100, n_equil=50, n_meas=100,
                    meta=dict(field="exp(GRF(0,0.8)) Matern nu=1.5 ell=20", gaps="50% uniform",
                              seed_field=seed, seed_mask=seed + 1))


def _batch64(seed=21, n_img=64, lmin=128, lmax=2048):
    rng = np.random.Generator(np.random.PCG64(seed))
    zs, gs, info = [], [], []
    for i in range(n_img):
        L = int(round(math.exp(rng.uniform(math.log(lmin), math.log(lmax)))))
        ell = float(rng.uniform(5.0, 40.0))
        lognormal = bool(rng.integers(0, 2))
        fs = int(rng.integers(0, 2**31 - 1))
        if lognormal:
            z = lognormal_grf((L, L), nu=0.5, ell=ell, log_mean=0.0, log_std=0.8, seed=fs)
        else:
            z = grf((L, L), nu=0.5, ell=ell, mean=50.0, std=10.0, seed=fs)
        frac = float(rng.uniform(0.3, 0.7))
        nrect = int(rng.integers(1, 6))
        cover = float(rng.uniform(0.05, 0.20))
        area = cover * L * L / nrect
        rects = []
        for _ in range(nrect):
            ar = float(rng.uniform(0.5, 2.0))
            h = max(1, min(L, int(round(math.sqrt(area * ar)))))
            w = max(1, min(L, int(round(area / h))))
            rects.append((int(rng.integers(0, L - h + 1)), int(rng.integers(0, L - w + 1)), h, w))
        m = block_gaps((L, L), rects)
        # top up with uniform gaps to reach the target fraction
        need = int(math.floor(frac * L * L)) - int(m.sum())
        if need > 0:
            free = np.flatnonzero(~m.ravel())
            pick = rng.permutation(free.size)[:need]
            mm = m.ravel()
            mm[free[pick]] = True
            m = mm.reshape(L, L)
        zs.append(z.astype(np.float32))
        gs.append(m.astype(np.uint8))
        info.append(dict(L=L, ell=ell, lognormal=lognormal, frac=float(m.mean()), rects=nrect))
    return Workload(f"batch{n_img}_ragged", zs, gs, chains=16, n_equil=50, n_meas=100,
                    meta=dict(images=info, seed=seed))


def _gamma8192(seed=31, L=8192, block=1024):
    z = gamma_grf((L, L), nu=0.5, ell=64.0, k=2.0, theta=10.0, seed=seed)
    g = uniform_gaps((L, L), 0.20, seed + 1)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    y0 = int(rng.integers(0, L - block + 1))
    x0 = int(rng.integers(0, L - block + 1))
    g[y0:y0 + block, x0:x0 + block] = True
    return Workload(f"gamma{L}_p20_block{block}", [z.astype(np.float32)], [g.astype(np.uint8)],
                    chains=32, n_equil=50, n_meas=100,
                    meta=dict(field="gamma(2,10) copula of exponential GRF ell=64",
                              gaps=f"20% uniform + {block}^2 block", block=(y0, x0, block)))


def _lognormal4096(seed=41, L=4096, frac=0.4):
    z = lognormal_grf((L, L), nu=0.5, ell=16.0, log_mean=5.0, log_std=1.0, seed=seed)
    g = uniform_gaps((L, L), frac, seed + 1)
    return Workload(f"lognormal{L}_p40", [z.astype(np.float32)], [g.astype(np.uint8)],
                    chains=32, n_equil=50, n_meas=100,
                    meta=dict(field="exp(GRF(5,1)) exponential ell=16", gaps="40% uniform",
                              seed_field=seed, seed_mask=seed + 1))


WORKLOADS = {
    "grf64": _grf64,
    "lognormal1024": _lognormal1024,
    "batch64": _batch64,
    "gamma8192": _gamma8192,
    "lognormal4096": _lognormal4096,
}


def workload(name: str, **kw) -> Workload:
    """Build a named workload; keyword arguments override its size parameters."""
    return WORKLOADS[name](**kw)
