"""FP64 CPU oracle of MPR gap filling (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its binding) never imports, links or calls it.

The arithmetic lives in ``mpr_oracle.c`` (plain C, double precision, written
from the paper's Sec. 2 and Algorithms 1-2); this module compiles it with gcc
on first use and exposes it through ctypes with numpy arrays.  See the C file
for the readings of the paper that it takes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmpr_oracle.so")
_lock = threading.Lock()
_lib = None

TWO_PI = 2.0 * np.pi
DIAG_FIELDS = ("r_minus_ap", "ap", "dH_over_T", "or_slack", "wrap_slack", "field",
               "sens", "accepted")


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (portable flags, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        u8 = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        u32 = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        i, d, u64, u32s, lng = C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_long
        dpn = C.c_void_p  # nullable double*
        sig = {
            "oracle_philox4x32_10": (None, [u32, u32, u32]),
            "oracle_map": (i, [i, i, dp, u8, dp, C.POINTER(d), C.POINTER(d)]),
            "oracle_unmap": (d, [d, d, d]),
            "oracle_hot_start": (None, [i, i, u8, dp, u64, u32s, u32s]),
            "oracle_sample_energy": (lng, [i, i, dp, u8, d, d, C.POINTER(d)]),
            "oracle_energy": (d, [i, i, dp, d, d]),
            "oracle_n_bonds": (lng, [i, i]),
            "oracle_torque": (None, [i, i, dp, d, d, dp]),
            "oracle_over_relax": (d, [d, dp, i, d, i, C.POINTER(d), C.POINTER(d)]),
            "oracle_sweep": (lng, [i, i, dp, u8, d, d, d, d, u64, u32s, u32s, u32s, i, dpn]),
            "oracle_site_update": (d, [d, dp, i, d, d, d, d, u64, u32s, u32s, u32s, i, i, i, i,
                                       C.POINTER(i), dpn]),
            "oracle_adapt_a": (d, [d, lng, lng, lng, d, d]),
            "oracle_e_of_T": (d, [i, i, i, i, d, d, d, d, d, u64, u32s, C.POINTER(d)]),
            "oracle_estimate_T": (i, [d, i, i, i, i, d, d, d, d, u64, u32s, d, d, d, i,
                                      C.POINTER(d)]),
            "oracle_simulate": (i, [i, i, dp, u8, d, d, d, d, d, i, i, i, i, i, u64, u32s,
                                    dp, dpn, dpn, dpn]),
            "oracle_sg_slope": (d, [dp, i]),
            "oracle_gmrf_energy": (d, [i, i, dp, d]),
            "oracle_gmrf_sample_energy": (lng, [i, i, dp, u8, d, C.POINTER(d)]),
            "oracle_gmrf_site_update": (d, [d, dp, i, d, d, d, u64, u32s, u32s, u32s, i, i, i,
                                            C.POINTER(i), dpn]),
            "oracle_gmrf_sweep": (lng, [i, i, dp, u8, d, d, d, u64, u32s, u32s, u32s, dpn]),
            "oracle_gmrf_simulate": (i, [i, i, dp, u8, d, d, d, d, i, i, i, u64, u32s, dp,
                                         C.POINTER(d)]),
            "oracle_equilibrate": (i, [i, i, dp, u8, d, d, d, d, d, i, i, i, i, u64, u32s, dp, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words and two key words -> four words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(c, k, out)
    return out


def map_to_angles(z, gap):
    """Eq. map on the sample sites -> (phi, z_min, z_max); gap sites hold 0."""
    lib = _load()
    z = _f64(z)
    g = _u8(gap)
    Ly, Lx = z.shape
    phi = np.zeros_like(z)
    zmin, zmax = C.c_double(), C.c_double()
    if lib.oracle_map(Lx, Ly, z, g, phi, C.byref(zmin), C.byref(zmax)) != 0:
        raise ValueError("degenerate sample range")
    return phi, zmin.value, zmax.value


def unmap(phi, zmin, zmax):
    """Inverse of Eq. map (Alg. 2 step 5.3), elementwise."""
    return zmin + (zmax - zmin) * np.asarray(phi, dtype=np.float64) / TWO_PI


def hot_start(phi, gap, seed, img, chain):
    """Copy of phi with gap angles drawn from U(0, 2 pi) (Alg. 2 step 1.8)."""
    lib = _load()
    out = _f64(phi).copy()
    g = _u8(gap)
    Ly, Lx = out.shape
    lib.oracle_hot_start(Lx, Ly, g, out, seed, img, chain)
    return out


def sample_energy(phi, gap, q=0.5, J=1.0):
    """Eq. mpr-sse over unordered sample-sample bonds -> (e_s, N_SP); e_s is nan if N_SP = 0."""
    lib = _load()
    p = _f64(phi)
    Ly, Lx = p.shape
    e = C.c_double(np.nan)
    nsp = lib.oracle_sample_energy(Lx, Ly, p, _u8(gap), q, J, C.byref(e))
    return e.value, int(nsp)


def energy(phi, q=0.5, J=1.0):
    """Total energy H of Eq. Hamiltonian_mod with open boundaries."""
    p = _f64(phi)
    Ly, Lx = p.shape
    return _load().oracle_energy(Lx, Ly, p, q, J)


def n_bonds(Lx, Ly):
    return int(_load().oracle_n_bonds(Lx, Ly))


def specific_energy(phi, q=0.5, J=1.0):
    p = _f64(phi)
    Ly, Lx = p.shape
    return energy(p, q, J) / n_bonds(Lx, Ly)


def torque(phi, q=0.5, J=1.0):
    """dH/dphi for every site."""
    p = _f64(phi)
    Ly, Lx = p.shape
    g = np.zeros_like(p)
    _load().oracle_torque(Lx, Ly, p, q, J, g)
    return g


def over_relax(phi, nbr, q=0.5, literal=False):
    """One over-relaxation step -> (phi', slack, field length)."""
    nb = _f64(nbr)
    slack, field = C.c_double(), C.c_double()
    out = _load().oracle_over_relax(float(phi), nb, nb.size, q, int(literal),
                                    C.byref(slack), C.byref(field))
    return out, slack.value, field.value


def sweep(phi, gap, *, T, a, seed, img=0, chain=0, sweep_index=0, q=0.5, J=1.0,
          literal_or=False, diagnostics=False):
    """One hybrid checkerboard sweep (Alg. 1) in place on a copy.

    Returns (phi_new, n_accepted) or (phi_new, n_accepted, diag) where diag is
    a dict of per-site arrays named in DIAG_FIELDS (nan on sample sites).
    """
    lib = _load()
    p = _f64(phi).copy()
    g = _u8(gap)
    Ly, Lx = p.shape
    d = None
    if diagnostics:
        d = np.full((Ly, Lx, len(DIAG_FIELDS)), np.nan)
    n_acc = lib.oracle_sweep(Lx, Ly, p, g, q, J, T, a, seed, img, chain, sweep_index,
                             int(literal_or), _ptr(d))
    if diagnostics:
        return p, int(n_acc), {k: d[..., j] for j, k in enumerate(DIAG_FIELDS)}
    return p, int(n_acc)


def site_update(phi, nbr, *, x, y, T, a, seed, img=0, chain=0, sweep_index=0, q=0.5, J=1.0,
                literal_or=False):
    """Alg. 1 on one site with neighbour angles nbr -> (phi_new, accepted, diag dict)."""
    nb = _f64(nbr)
    acc = C.c_int()
    d = np.zeros(len(DIAG_FIELDS))
    out = _load().oracle_site_update(float(phi), nb, nb.size, q, J, T, a, seed, img, chain,
                                     sweep_index, int(x), int(y), (int(x) + int(y)) & 1,
                                     int(literal_or), C.byref(acc), _ptr(d))
    return out, bool(acc.value), dict(zip(DIAG_FIELDS, d))


def adapt_a(a, n_acc, n_gap, i, A_targ=0.3, k_a=3.0):
    return _load().oracle_adapt_a(a, n_acc, n_gap, i, A_targ, k_a)


def e_of_T(T, *, L, K, n_eq, n_meas, seed, img=0, q=0.5, J=1.0, A_targ=0.3, k_a=3.0):
    """Equilibrium specific energy e(T, L) by unconditional simulation -> (mean, variance)."""
    var = C.c_double()
    m = _load().oracle_e_of_T(L, K, n_eq, n_meas, q, J, T, A_targ, k_a, seed, img, C.byref(var))
    return m, var.value


def estimate_T(e_s, *, L, K, n_eq, n_meas, seed, img=0, q=0.5, J=1.0, A_targ=0.3, k_a=3.0,
               T_lo=1e-5, T_hi=20.0, rel_tol=1e-3, max_iter=60):
    """SEM temperature T_hat = e^-1(e_s | L) by bisection (Sec. 2.3)."""
    T = C.c_double()
    rc = _load().oracle_estimate_T(e_s, L, K, n_eq, n_meas, q, J, A_targ, k_a, seed, img,
                                   T_lo, T_hi, rel_tol, max_iter, C.byref(T))
    if rc != 0:
        raise ValueError("sample specific energy outside the range of e(T)")
    return T.value


def simulate(phi_s, gap, *, T, R, n_equil, n_meas, seed, img=0, q=0.5, J=1.0, A_targ=0.3,
             k_a=3.0, freeze_a=True, literal_or=False, history=False):
    """Alg. 2 at fixed T over R chains -> dict(phi_mean, [e_hist, a, acc_hist])."""
    lib = _load()
    p = _f64(phi_s)
    g = _u8(gap)
    Ly, Lx = p.shape
    mean = np.zeros_like(p)
    n_sw = n_equil + n_meas
    eh = np.zeros((R, n_sw)) if history else None
    ah = np.zeros(R) if history else None
    acch = np.zeros((R, n_sw)) if history else None
    lib.oracle_simulate(Lx, Ly, p, g, q, J, T, A_targ, k_a, R, n_equil, n_meas,
                        int(freeze_a), int(literal_or), seed, img, mean,
                        _ptr(eh), _ptr(ah), _ptr(acch))
    out = dict(phi_mean=mean)
    if history:
        out.update(e_hist=eh, a=ah, acc_hist=acch)
    return out


def fill(z, gap, *, R, n_equil, n_meas, seed, img=0, T=None, sem=None, q=0.5, J=1.0,
         A_targ=0.3, k_a=3.0, freeze_a=True):
    """Whole gap fill of one image (Alg. 2): map, e_s, SEM T (unless given), simulate, unmap.

    ``sem`` holds the keyword arguments of estimate_T (L, K, n_eq, n_meas).
    Returns dict(z_hat, T, e_s, zmin, zmax).
    """
    phi, zmin, zmax = map_to_angles(z, gap)
    e_s, nsp = sample_energy(phi, gap, q, J)
    if T is None:
        if nsp == 0:
            raise ValueError("no sample pairs")
        T = estimate_T(e_s, seed=seed, img=img, q=q, J=J, A_targ=A_targ, k_a=k_a, **sem)
    sim = simulate(phi, gap, T=T, R=R, n_equil=n_equil, n_meas=n_meas, seed=seed, img=img,
                   q=q, J=J, A_targ=A_targ, k_a=k_a, freeze_a=freeze_a)
    z_hat = np.where(np.asarray(gap) != 0, unmap(sim["phi_mean"], zmin, zmax),
                     np.asarray(z, dtype=np.float64))
    return dict(z_hat=z_hat, T=T, e_s=e_s, zmin=zmin, zmax=zmax)


def select_q(z, gap, holdout, qs, *, R, n_equil, n_meas, seed, sem, img=0, J=1.0,
             A_targ=0.3, k_a=3.0, freeze_a=True):
    """Cross-validated choice of the modification factor q (the conclusions name the
    selection of q in (0, 1/2] by cross-validation as an extension of the method).

    Steps, for every candidate q in ``qs`` (each in (0, 1/2]):
      1. the samples flagged in ``holdout`` are set aside as a validation set, as in
         Sec. 3's validation design: they become gaps next to the image's own gaps,
         and the angle map uses the extremes of the remaining samples;
      2. the whole gap fill of Alg. 2 at that q: sample specific energy of the
         remaining samples, SEM temperature (Sec. 2.3), conditional simulation of R
         realisations with the same seed for every q, realisation mean, back-transform;
      3. the score is the absolute error averaged over the validation points (AAE of
         Sec. 3) of that prediction.
    The chosen q is the first candidate with the smallest score.  A candidate whose
    sample specific energy lies outside the range of e(T) scores infinity (T = nan).
    A holdout flag on a gap pixel is ignored.  Returns dict(q, scores, T).
    """
    z = np.asarray(z, dtype=np.float64)
    g = np.asarray(gap) != 0
    hold = (np.asarray(holdout) != 0) & ~g
    if not hold.any():
        raise ValueError("no held-out sample")
    g_cv = (g | hold).astype(np.uint8)
    scores, Ts = [], []
    for q in qs:
        if not 0.0 < q <= 0.5:
            raise ValueError("q must lie in (0, 1/2]")
        try:
            r = fill(z, g_cv, R=R, n_equil=n_equil, n_meas=n_meas, seed=seed, img=img, sem=sem,
                     q=q, J=J, A_targ=A_targ, k_a=k_a, freeze_a=freeze_a)
        except ValueError:
            # e_s outside the range of e(T) at this q: no SEM temperature exists
            scores.append(math.inf)
            Ts.append(math.nan)
            continue
        scores.append(float(np.mean(np.abs(r["z_hat"][hold] - z[hold]))))
        Ts.append(r["T"])
    if not np.isfinite(scores).any():
        raise ValueError("no candidate q has a SEM temperature")
    k = int(np.argmin(scores))
    return dict(q=float(qs[k]), scores=np.array(scores), T=np.array(Ts))


def sg_slope(y):
    """Least-squares slope of a series against its index (degree-1 Savitzky-Golay)."""
    y = _f64(y)
    return _load().oracle_sg_slope(y, y.size)


def equilibrate(phi_s, gap, *, T, R, seed, img=0, n_f=5, n_fit=20, i_max=500, q=0.5, J=1.0,
                A_targ=0.3, k_a=3.0):
    """Alg. 2 step 4 with the slope stop for R chains -> (sweeps run, chain-mean energies, states)."""
    p = _f64(phi_s)
    g = _u8(gap)
    Ly, Lx = p.shape
    out = np.zeros((R, Ly, Lx))
    em = np.zeros(i_max + 1)
    n = _load().oracle_equilibrate(Lx, Ly, p, g, q, J, T, A_targ, k_a, R, n_f, n_fit, i_max,
                                   seed, img, out, em)
    return int(n), em[:n], out


# ------------------------------------------------------------ GMRF (Sec. 4.3)

def gmrf_energy(phi, J=1.0):
    """H = J sum_<ij> (dphi^2 / (2 pi^2) - 1) of the GMRF pair interaction."""
    p = _f64(phi)
    Ly, Lx = p.shape
    return _load().oracle_gmrf_energy(Lx, Ly, p, J)


def gmrf_sample_energy(phi, gap, J=1.0):
    p = _f64(phi)
    Ly, Lx = p.shape
    e = C.c_double(np.nan)
    n = _load().oracle_gmrf_sample_energy(Lx, Ly, p, _u8(gap), J, C.byref(e))
    return e.value, int(n)


def gmrf_sweep(phi, gap, *, T, a, seed, img=0, chain=0, sweep_index=0, J=1.0, diagnostics=False):
    p = _f64(phi).copy()
    Ly, Lx = p.shape
    d = np.full((Ly, Lx, len(DIAG_FIELDS)), np.nan) if diagnostics else None
    n = _load().oracle_gmrf_sweep(Lx, Ly, p, _u8(gap), J, T, a, seed, img, chain, sweep_index,
                                  _ptr(d))
    if diagnostics:
        return p, int(n), {k: d[..., j] for j, k in enumerate(DIAG_FIELDS)}
    return p, int(n)


def gmrf_simulate(phi_s, gap, *, T, R, n_equil, n_meas, seed, img=0, J=1.0, A_targ=0.3, k_a=3.0):
    p = _f64(phi_s)
    Ly, Lx = p.shape
    mean = np.zeros_like(p)
    em = C.c_double()
    _load().oracle_gmrf_simulate(Lx, Ly, p, _u8(gap), J, T, A_targ, k_a, R, n_equil, n_meas, seed,
                                 img, mean, C.byref(em))
    return dict(phi_mean=mean, e_mean=em.value)
