"""Writes lognormal256_longrun.json: the oracle's long-run statistics on a 256 x 256
field shaped like the 1024 x 1024 lognormal workload (exp of a GRF with log-mean 0,
log-std 0.8, Whittle-Matern nu = 1.5, correlation length 20 px; 50% of the pixels
removed uniformly at random).

Everything here comes from `oracle/` (FP64) and the seeded input generators; nothing
from the CUDA path.  Stored:

* e_s, the sample specific energy, and T_sem, the SEM temperature: the root of
  e(T, L) = e_s by bisection on an unconditional L = 256 lattice (Sec. 2.3);
* at T_sem, 100 independent realisations (Alg. 2, hot start, 100 equilibration and
  100 measurement sweeps): the mean specific energy of each realisation over its
  measurement sweeps, and the MAE / RMSE of the realisation mean against the removed
  values (Sec. 4.1's error measures).

The 100 realisations are ten blocks of ten chains that differ in their seed, so
that the blocks run in parallel; chains of different seeds draw independent random
streams.  Run from the repository root:  python tests/golden/make_longrun_lognormal256.py
(about ten minutes on eight cores).
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "lognormal256_longrun.json")
SIDE = 256
BLOCKS, CHAINS = 10, 10
N_EQUIL, N_MEAS = 100, 100
SEED_T = 0x7A11
SEED_SIM = 0x5A3E00
SEM = dict(L=256, K=4, n_eq=150, n_meas=150, T_lo=1e-4, T_hi=1.0, rel_tol=1e-3)


def _input():
    import synthetic
    w = synthetic.workload("lognormal1024", L=SIDE)
    return w.z[0].astype(np.float64), w.gap[0]


def _estimate(e_s):
    import oracle
    return oracle.estimate_T(e_s, seed=SEED_T, **SEM)


def _block(args):
    k, T = args
    import oracle
    z, g = _input()
    phi, _, _ = oracle.map_to_angles(z, g)
    sim = oracle.simulate(phi, g, T=T, R=CHAINS, n_equil=N_EQUIL, n_meas=N_MEAS,
                          seed=SEED_SIM + k, history=True)
    return sim["phi_mean"], sim["e_hist"][:, N_EQUIL:].mean(axis=1)


def main():
    import oracle
    oracle.build()
    z, g = _input()
    phi, zmin, zmax = oracle.map_to_angles(z, g)
    e_s, n_sp = oracle.sample_energy(phi, g)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(os.cpu_count() or 1, BLOCKS)) as pool:
        T = pool.apply(_estimate, (e_s,))
        # the root must lie inside the bracket, not at one of its ends
        assert SEM["T_lo"] * 1.01 < T < SEM["T_hi"] / 1.01, T
        res = pool.map(_block, [(k, T) for k in range(BLOCKS)])
    phi_mean = np.mean([r[0] for r in res], axis=0)
    e_chain = np.concatenate([r[1] for r in res])
    z_hat = oracle.unmap(phi_mean, zmin, zmax)
    m = g == 1
    err = z_hat[m] - z[m]
    rec = {
        "input": {"workload": "lognormal1024", "side": SIDE, "gap_fraction": float(m.mean())},
        "e_s": float(e_s), "n_sp": int(n_sp),
        "sem": {**SEM, "seed": SEED_T, "T": float(T)},
        "simulate": {"blocks": BLOCKS, "chains_per_block": CHAINS, "seed0": SEED_SIM,
                     "n_equil": N_EQUIL, "n_meas": N_MEAS, "freeze_a": True},
        "e_chain_mean": [float(v) for v in e_chain],
        "mae": float(np.mean(np.abs(err))), "rmse": float(np.sqrt(np.mean(err ** 2))),
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: rec[k] for k in ("e_s", "mae", "rmse")}), rec["sem"]["T"])


if __name__ == "__main__":
    main()
