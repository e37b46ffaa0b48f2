"""Full-size parity on the workloads' own sizes, in the benchmark's launch configuration.

The oracle cannot sweep these grids, so each test checks sampled outputs the
oracle computes one by one: after one GPU sweep, a random sample of red gap
sites is recomputed by the oracle's single-site update (Alg. 1) from the
state before the sweep, and a random sample of black gap sites from the
state after the red half (their neighbours are red).  The decision-parity
rule of tests/parity.py applies: angles within 1e-5 rad unless the oracle's
decision lay within tolerance of its threshold (Metropolis: 1e-6), those
counted and kept at or below 1e-4 of the sampled sites.  Whole-grid properties are checked too: sample pixels
never move, gap angles stay in [0, 2 pi), the recorded energy equals the
energy of the state, predictions at sample pixels return the data.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic
from parity import Tally

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1710_03038_gb300 as mpr  # noqa: E402

SEED = 0xFACE5EED
N_SAMPLE = 400


def _neighbours(st, y, x):
    Ly, Lx = st.shape
    out = []
    if y > 0:
        out.append(st[y - 1, x])
    if y + 1 < Ly:
        out.append(st[y + 1, x])
    if x > 0:
        out.append(st[y, x - 1])
    if x + 1 < Lx:
        out.append(st[y, x + 1])
    return out


def _check_sampled_sweep(ctx, gaps, T, rng):
    """One GPU sweep; sampled red/black sites against the oracle's site update."""
    before = [s.clone() for s in ctx.get_state()]
    a = ctx.chain_info()["a"]
    sweep_idx, _ = ctx.sweep_index()
    ctx.sweep(1, "equil", record_energy=True)
    after = ctx.get_state()
    info = ctx.chain_info()
    tally = Tally()
    for i, g in enumerate(gaps):
        R = before[i].shape[0]
        Ly, Lx = g.shape
        gy, gx = np.nonzero(g)
        red = ((gy + gx) & 1) == 0
        for colour, sel in ((0, red), (1, ~red)):
            idx = np.flatnonzero(sel)
            pick = rng.choice(idx, size=min(N_SAMPLE // len(gaps) + 1, idx.size), replace=False)
            chains = rng.integers(0, R, size=pick.size)
            for p, c in zip(pick, chains):
                y, x = int(gy[p]), int(gx[p])
                # red sites see the state before the sweep, black sites the red half
                src = before[i][c] if colour == 0 else after[i][c]
                ys = slice(max(y - 1, 0), min(y + 2, Ly))
                xs = slice(max(x - 1, 0), min(x + 2, Lx))
                patch = src[ys, xs].double().cpu().numpy()
                nb = _neighbours(patch, y - ys.start, x - xs.start)
                phi0 = float(before[i][c, y, x])
                ref, _, diag = oracle.site_update(phi0, nb, x=x, y=y, T=float(T[i]),
                                                  a=float(a[i, c]), seed=SEED, img=i, chain=int(c),
                                                  sweep_index=sweep_idx)
                tally.check_site(ref, float(after[i][c, y, x]), diag)
        # sample pixels never move, gap angles stay in [0, 2 pi)
        gm = torch.from_numpy(g.astype(bool)).cuda()
        assert torch.equal(after[i][:, ~gm], before[i][:, ~gm])
        ga = after[i][:, gm]
        assert bool((ga >= 0).all()) and bool((ga < 2 * math.pi + 1e-6).all())
    tally.assert_budget()
    print(tally)
    return info


def _run(name, T=None, tune=None, **kw):
    w = synthetic.workload(name, **kw)
    zs = [torch.from_numpy(z).cuda() for z in w.z]
    gs = [torch.from_numpy(g).cuda() for g in w.gap]
    ctx = mpr.Context(zs, gs, chains=w.chains, params=mpr.Params(seed=SEED))
    if T is None:
        T = ctx.estimate_T()
    else:
        ctx.set_T(T)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (len(zs),))
    ctx.sweep(2, "equil")
    rng = np.random.default_rng(7)
    info = _check_sampled_sweep(ctx, w.gap, T, rng)
    e = ctx.energy()
    assert np.max(np.abs(info["e_last"] - e)) < 2e-6, np.max(np.abs(info["e_last"] - e))
    ctx.sweep(3, "measure")
    zh = ctx.predict()
    for z, g, p in zip(w.z, w.gap, zh):
        p = p.cpu().numpy()
        m = g == 0
        assert np.array_equal(p[m], z[m])
        zmin, zmax = z[m].min(), z[m].max()
        assert np.all(p[~m] >= zmin - 1e-3 * abs(zmin)) and np.all(p[~m] <= zmax * (1 + 1e-6))
    return ctx, T


def test_fullsize_lognormal1024_100_chains():
    _run("lognormal1024")


def test_fullsize_batch64_ragged():
    _run("batch64")


def test_fullsize_lognormal4096_32_chains():
    ctx, T = _run("lognormal4096")
    assert 1e-5 < T[0] < 1.0


def test_fullsize_gamma8192_block_gap():
    _run("gamma8192")


def test_autograd_on_512_crop_of_the_4096_field():
    """Energy autograd on a 512^2 crop of the 4096^2 lognormal field (32 realisations):
    torque and dH/dJ against central differences (h = 1e-3, FP64) and the oracle's gradient."""
    w = synthetic.workload("lognormal4096")
    z = torch.from_numpy(w.z[0]).cuda()
    g = torch.from_numpy(w.gap[0]).cuda()
    ctx = mpr.Context([z], [g], chains=32, params=mpr.Params(seed=SEED))
    ctx.set_T([3e-3])
    ctx.sweep(5, "equil")
    crop = ctx.get_state()[0][:4, 1000:1512, 2000:2512].contiguous()  # 4 realisations
    phi = crop.clone().requires_grad_(True)
    J = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    H = mpr.MPREnergy.apply(phi, J)
    wts = torch.tensor([1.0, -0.5, 0.25, 2.0], dtype=torch.float64, device="cuda")
    (H * wts).sum().backward()
    rng = np.random.default_rng(11)
    for k in range(4):
        p64 = crop[k].double().cpu().numpy()
        assert abs(H[k].item() - oracle.energy(p64)) < 1e-6 * abs(H[k].item())
        gk = phi.grad[k].cpu().numpy()
        assert np.max(np.abs(gk - wts[k].item() * oracle.torque(p64))) < 2e-5
        for _ in range(6):
            y, x = int(rng.integers(0, 512)), int(rng.integers(0, 512))
            e_p = p64.copy(); e_p[y, x] += 1e-3
            e_m = p64.copy(); e_m[y, x] -= 1e-3
            fd = (oracle.energy(e_p) - oracle.energy(e_m)) / 2e-3 * wts[k].item()
            assert abs(gk[y, x] - fd) < 1e-5
    dJ = sum(wts[k].item() * oracle.energy(crop[k].double().cpu().numpy()) for k in range(4))
    assert abs(J.grad.item() - dJ) < 1e-6 * abs(dJ)


def test_newton_T_matches_oracle_bisection_on_4096_field():
    """SEM on the 4096^2 field's e_s: GPU Newton steps vs the oracle's bisection within 1%."""
    w = synthetic.workload("lognormal4096")
    z = torch.from_numpy(w.z[0]).cuda()
    g = torch.from_numpy(w.gap[0]).cuda()
    topts = mpr.TOpts(L=64, chains=8, n_equil=60, n_meas=120, iters=6)
    ctx = mpr.Context([z], [g], chains=2, params=mpr.Params(seed=SEED), topts=topts)
    T_gpu = ctx.estimate_T()[0]
    e_s = ctx.image_info()["e_s"][0]
    T_or = oracle.estimate_T(e_s, L=64, K=4, n_eq=150, n_meas=150, seed=SEED, rel_tol=2e-3)
    assert abs(T_gpu - T_or) < 0.01 * T_or, (T_gpu, T_or)
