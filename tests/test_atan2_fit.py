"""The colour pass's own atan2 polynomial, checked on the CPU.

atan(t) for t in [0, 1] is approximated by t P(t^2), P of degree 7 (an odd
polynomial of degree 15), with the coefficients written in the CUDA source.
The test reads them from there and checks them against the minimax
approximation computed here by the Remez exchange (equioscillating error at
9 alternation points): the committed coefficients, rounded to FP32, must lie
within their rounding of the minimax error level, and the FP32 Horner scheme
the kernel uses must stay within 1.3e-7 rad.
"""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEG = 7  # degree of P in t^2


def _coefficients():
    src = open(os.path.join(ROOT, "paper_1710_03038_gb300", "csrc", "mpr_device.cuh")).read()
    body = src[src.index("atan2_pair("):]
    body = body[:body.index("float2 r = mul2(p, t);")]
    c = [float(v) for v in re.findall(r"f2\((-?[0-9.]+)f\)", body)]
    assert len(c) == DEG + 1, c  # t^15 ... t^1, Horner order
    return c


def _horner(c, t):
    t2 = t * t
    p = np.full_like(t, c[0])
    for k in c[1:]:
        p = p * t2 + k
    return t * p


def remez_atan(iters=30):
    """Minimax t P(t^2) ~ atan(t) on [0, 1] (absolute error): returns the
    coefficients (highest first) and the levelled error E."""
    n = DEG + 2  # unknowns: DEG + 1 coefficients and E
    grid = np.linspace(0.0, 1.0, 400001)
    # start from Chebyshev-like points, away from t = 0 where the error vanishes
    ref = 0.5 - 0.5 * np.cos(np.pi * (np.arange(n) + 0.5) / n)
    E = 0.0
    for _ in range(iters):
        A = np.zeros((n, n))
        for k in range(DEG + 1):  # column k: t^(2k+1)
            A[:, k] = ref ** (2 * k + 1)
        A[:, DEG + 1] = (-1.0) ** np.arange(n)
        sol = np.linalg.solve(A, np.arctan(ref))
        low_first, E = sol[:DEG + 1], sol[DEG + 1]
        c = low_first[::-1]
        err = _horner(c, grid) - np.arctan(grid)
        # new reference: the extreme of each run of one error sign
        sgn = np.sign(err)
        sgn[sgn == 0] = 1
        cuts = np.flatnonzero(np.diff(sgn)) + 1
        runs = np.split(np.arange(grid.size), cuts)
        ext = np.array([r[np.argmax(np.abs(err[r]))] for r in runs if r.size])
        if ext.size < n:
            break
        # keep n alternating extremes with the largest errors
        while ext.size > n:
            drop = 0 if abs(err[ext[0]]) < abs(err[ext[-1]]) else ext.size - 1
            ext = np.delete(ext, drop)
        ref = grid[ext]
    return c, abs(E)


def test_atan_polynomial_is_the_minimax_fit_rounded_to_fp32():
    c_opt, E = remez_atan()
    t = np.linspace(0.0, 1.0, 2_000_001)
    e_opt = np.max(np.abs(_horner(c_opt, t) - np.arctan(t)))
    # the exchange levelled the error: its maximum is the levelled value
    assert abs(e_opt - E) < 0.05 * E, (e_opt, E)
    assert 3.0e-8 < E < 4.5e-8, E
    c = _coefficients()
    err = np.max(np.abs(_horner(c, t) - np.arctan(t)))
    # rounding each coefficient to FP32 moves t P(t^2) by at most sum |c_k| ulp/2
    rounding = sum(abs(k) * 2.0 ** -24 for k in c)
    assert err <= E + rounding, (err, E, rounding)
    assert err < 6.5e-8, err
    # and the committed coefficients are those of the minimax fit, rounded
    assert np.allclose(c, c_opt, rtol=0, atol=2e-6), (c, c_opt)


def test_atan_polynomial_in_fp32_horner():
    c = [np.float32(v) for v in _coefficients()]
    t = np.linspace(0.0, 1.0, 200_001).astype(np.float32)
    t2 = (t * t).astype(np.float32)
    p = np.full_like(t, c[0])
    for k in c[1:]:
        # the kernel's FMA: one rounding of p * t2 + k
        p = (p.astype(np.float64) * t2.astype(np.float64) + np.float64(k)).astype(np.float32)
    r = (p * t).astype(np.float32)
    err = r.astype(np.float64) - np.arctan(t.astype(np.float64))
    assert np.max(np.abs(err)) < 1.3e-7, np.max(np.abs(err))
