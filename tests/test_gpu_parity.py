"""Parity of the CUDA path against the FP64 oracle (needs a GPU).

Sweep-by-sweep parity: the GPU and the oracle start every sweep from the same
state (the oracle's, rounded to FP32), the same random stream and the same a,
T, under the decision-parity rule of tests/parity.py: angles within 1e-5 rad
except where a decision lay within tolerance of its threshold (Metropolis:
1e-6), those counted and kept at or below 1e-4 of the sites.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synthetic
from parity import Tally

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1710_03038_gb300 as mpr  # noqa: E402

TWO_PI = 2 * math.pi
SEED = 0x5EED1234ABCD


def compare_sweep(before, after_gpu, gap, tally, *, T, a, seed, img, chain, sweep_index,
                  **kw):
    """The oracle's sweep of one realisation from the GPU's starting state, checked
    with the decision-parity rule; returns (oracle state, oracle accepts, sites that
    may differ)."""
    ref, n_acc, diag = oracle.sweep(before.astype(np.float64), gap, T=T, a=float(a), seed=seed,
                                    img=img, chain=chain, sweep_index=sweep_index,
                                    diagnostics=True, **kw)
    n_diff = tally.check_grid(ref, after_gpu, gap, diag)
    # sample sites never move
    assert np.array_equal(after_gpu[gap == 0], before[gap == 0])
    return ref, n_acc, n_diff


def ragged_images():
    shapes = [(64, 64), (37, 53), (70, 31), (5, 130)]
    zs, gs = [], []
    for k, (h, w) in enumerate(shapes):
        z = synthetic.grf((h, w), nu=0.5, ell=6.0, mean=50, std=10, seed=100 + k)
        g = synthetic.uniform_gaps((h, w), 0.25 + 0.15 * k, 200 + k)
        zs.append(z.astype(np.float32))
        gs.append(g.astype(np.uint8))
    # one image with a block gap
    gs[0][10:30, 20:44] = 1
    return zs, gs


def make_ctx(zs, gs, chains, path="tiled", **kw):
    return mpr.Context(zs, gs, chains=chains, params=mpr.Params(seed=SEED, path=path, **kw))


# ------------------------------------------------------------------ RNG

def test_philox_matches_known_answers_and_toolkit(golden_dir):
    rows = []
    with open(f"{golden_dir}/philox4x32_10_kat.txt") as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    for r in rows:
        out = mpr.philox(np.array([r[0:4]], dtype=np.uint32), r[4:6])
        assert list(out[0]) == r[6:10]
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = [0xDEADBEEF, 0x12345678]
    mine = mpr.philox(ctr, key)
    ref = mpr.philox(ctr, key, reference=True)
    assert np.array_equal(mine, ref)
    o = np.array([oracle.philox4x32_10(c, key) for c in ctr[:64]])
    assert np.array_equal(mine[:64], o)


def test_own_math_against_cuda_routines():
    """The library's atan2 and series sine against CUDA atan2f / sinf and FP64."""
    g = torch.Generator(device="cpu").manual_seed(0)
    y = (torch.rand(200000, generator=g) * 8 - 4).cuda()
    x = (torch.rand(200000, generator=g) * 8 - 4).cuda()
    mine = mpr.math_probe(0, y, x).double().cpu().numpy()
    cuda = mpr.math_probe(1, y, x).double().cpu().numpy()
    exact = np.arctan2(y.double().cpu().numpy(), x.double().cpu().numpy())
    assert np.max(np.abs(mine - exact)) < 4e-7
    assert np.max(np.abs(mine - cuda)) < 5e-7
    t = (torch.rand(200000, generator=g) * math.pi - math.pi / 2).cuda()
    t[:3] = torch.tensor([1e-6, -3e-4, 0.0])
    s_mine = mpr.math_probe(2, t).double().cpu().numpy()
    s_cuda = mpr.math_probe(3, t).double().cpu().numpy()
    s_exact = np.sin(t.double().cpu().numpy())
    rel = np.abs(s_mine - s_exact) / np.maximum(np.abs(s_exact), 1e-30)
    assert np.max(rel[np.abs(s_exact) > 0]) < 3e-7
    assert np.max(np.abs(s_mine - s_cuda)) < 3e-7


# ------------------------------------------------------------- init

@pytest.mark.parametrize("path", ["tiled", "plain"])
def test_init_map_hot_start_and_sample_energy(path):
    zs, gs = ragged_images()
    R = 3
    ctx = make_ctx(zs, gs, R, path)
    info = ctx.image_info()
    st = [s.cpu().numpy() for s in ctx.get_state()]
    for i, (z, g) in enumerate(zip(zs, gs)):
        phi, zmin, zmax = oracle.map_to_angles(z.astype(np.float64), g)
        assert info["zmin"][i] == zmin and info["zmax"][i] == zmax
        assert info["n_gap"][i] == g.sum()
        e_s, nsp = oracle.sample_energy(phi, g)
        assert info["n_sp"][i] == nsp
        assert abs(info["e_s"][i] - e_s) < 1e-6
        for c in range(R):
            ref = oracle.hot_start(phi, g, SEED, i, c)
            assert np.max(np.abs(st[i][c] - ref)) < 1e-6


# ---------------------------------------------------- sweep by sweep

@pytest.mark.parametrize("path", ["tiled", "plain"])
def test_sweep_by_sweep_parity_ragged_batch(path):
    zs, gs = ragged_images()
    R = 3
    ctx = make_ctx(zs, gs, R, path)
    T = np.array([0.15, 0.3, 0.08, 0.5])
    ctx.set_T(T)
    state = [s.cpu().numpy().astype(np.float64) for s in ctx.get_state()]
    tally = Tally()
    a_vals = ctx.chain_info()["a"]
    for k in range(6):
        ctx.set_state([s.astype(np.float32) for s in state])
        before = [s.astype(np.float32) for s in state]
        sweep_idx, eq_idx = ctx.sweep_index()
        ctx.sweep(1, "equil", record_energy=True)
        after = [s.cpu().numpy() for s in ctx.get_state()]
        info = ctx.chain_info()
        for i, g in enumerate(gs):
            for c in range(R):
                ref, n_acc, n_diff = compare_sweep(
                    before[i][c], after[i][c], g, tally, T=T[i], a=a_vals[i, c], seed=SEED,
                    img=i, chain=c, sweep_index=sweep_idx)
                assert abs(int(info["accepted"][i, c]) - n_acc) <= n_diff
                # the a-adaptation (Alg. 2 step 4.2) from the GPU's own count
                a_ref = oracle.adapt_a(float(a_vals[i, c]), int(info["accepted"][i, c]),
                                       int(g.sum()), eq_idx)
                assert abs(info["a"][i, c] - a_ref) < 1e-6 * a_ref
                # energy recorded after the sweep vs the oracle energy of the GPU state
                e_ref = oracle.specific_energy(after[i][c].astype(np.float64))
                assert abs(info["e_last"][i, c] - e_ref) < 2e-6
                state[i][c] = ref
        a_vals = info["a"]
    tally.assert_budget()
    print(tally)


@pytest.mark.parametrize("path,R,cg", [("tiled", 4, 0), ("plain", 4, 0), ("tiled", 8, 4)])
@pytest.mark.parametrize("freeze_a", [True, False])
def test_measurement_sweeps_match_oracle_state_by_state(path, R, cg, freeze_a):
    """Alg. 2 step 5 from a shared state: three sampling sweeps, each against the
    oracle's sweep with the a that step 5.2 prescribes (the frozen equilibration a,
    or a = 1 as printed); a and the equilibration index stay put; the realisation
    sums equal the sums of the GPU's own states (FP32 partial sums) and the oracle's
    states wherever no decision flipped; the prediction and its spread follow from
    the sums.  With 8 chains in groups of 4 two blocks of the tiled pass add to
    each site's sums."""
    zs, gs = ragged_images()
    ctx = make_ctx(zs, gs, R, path, freeze_a_in_measure=freeze_a, chain_group=cg)
    T = np.array([0.15, 0.3, 0.08, 0.5])
    ctx.set_T(T)
    ctx.sweep(4, "equil")
    a0 = ctx.chain_info()["a"]
    _, eq0 = ctx.sweep_index()
    ctx.reset_accumulators()
    state = [s.cpu().numpy().astype(np.float64) for s in ctx.get_state()]
    gsum = [np.zeros(g.shape) for g in gs]
    gsum2 = [np.zeros(g.shape) for g in gs]
    osum = [np.zeros(g.shape) for g in gs]
    differs = [np.zeros(g.shape, bool) for g in gs]
    tally = Tally()
    for k in range(3):
        ctx.set_state([s.astype(np.float32) for s in state])
        before = [s.astype(np.float32) for s in state]
        s_idx, _ = ctx.sweep_index()
        ctx.sweep(1, "measure")
        after = [s.cpu().numpy() for s in ctx.get_state()]
        info = ctx.chain_info()
        assert np.array_equal(info["a"], a0)
        assert ctx.sweep_index()[1] == eq0
        for i, g in enumerate(gs):
            for c in range(R):
                a_use = float(a0[i, c]) if freeze_a else 1.0
                ref, _, diag = oracle.sweep(before[i][c].astype(np.float64), g, T=T[i], a=a_use,
                                            seed=SEED, img=i, chain=c, sweep_index=s_idx,
                                            diagnostics=True)
                _, m = tally.check_grid(ref, after[i][c], g, diag, mask=True)
                differs[i] |= m
                gsum[i] += after[i][c]
                gsum2[i] += after[i][c].astype(np.float64) ** 2
                osum[i] += ref
                state[i][c] = ref
    tally.assert_budget()
    print(tally)
    s1, s2, n = ctx.accumulators()
    assert n == 3 * R
    for i, g in enumerate(gs):
        m = g == 1
        a1 = s1[i].cpu().numpy()
        a2 = s2[i].cpu().numpy()
        assert np.all(a1[~m] == 0) and np.all(a2[~m] == 0)
        # the sums the kernels formed, against the states they produced
        assert np.allclose(a1[m], gsum[i][m], rtol=1e-6, atol=1e-5)
        assert np.allclose(a2[m], gsum2[i][m], rtol=1e-6, atol=1e-4)
        # against the oracle's states where every decision agreed
        ok = m & ~differs[i]
        assert np.all(np.abs(a1[ok] - osum[i][ok]) <= 3 * R * 1e-5 + 1e-5 * np.abs(osum[i][ok]))
    zh, zs_ = ctx.predict(std=True)
    zh_only = ctx.predict(std=False)
    info = ctx.image_info()
    for i, (z, g) in enumerate(zip(zs, gs)):
        m = g == 1
        zmin, zmax = float(info["zmin"][i]), float(info["zmax"][i])
        mean = s1[i].cpu().numpy()[m] / n
        var = np.maximum(s2[i].cpu().numpy()[m] / n - mean ** 2, 0.0)
        want = zmin + (zmax - zmin) * mean / TWO_PI
        assert np.allclose(zh[i].cpu().numpy()[m], want, rtol=1e-6, atol=1e-4)
        assert np.array_equal(zh[i].cpu().numpy(), zh_only[i].cpu().numpy())
        assert np.allclose(zs_[i].cpu().numpy()[m], (zmax - zmin) * np.sqrt(var) / TWO_PI,
                           rtol=1e-4, atol=1e-3)
        assert np.array_equal(zh[i].cpu().numpy()[~m], z[~m])


def test_accumulators_round_trip_resumes_sampling():
    """Checkpoint of a sampling run through the accumulator and state access: a
    context restored from them continues exactly as the original."""
    zs, gs = ragged_images()
    R = 4
    outs = []
    ref = make_ctx(zs, gs, R)
    ref.set_T([0.2, 0.2, 0.1, 0.4])
    ref.sweep(3, "equil")
    ref.sweep(2, "measure")
    saved = ([s.clone() for s in ref.get_state()], ref.accumulators(), ref.sweep_index(),
             ref.chain_info()["a"])
    ref.sweep(2, "measure")
    want = [p.cpu().numpy() for p in ref.predict()]
    ctx = make_ctx(zs, gs, R)
    ctx.set_T([0.2, 0.2, 0.1, 0.4])
    ctx.set_state(saved[0])
    s1, s2, n = saved[1]
    ctx.set_accumulators(s1, s2, n)
    ctx.set_sweep_index(*saved[2])
    ctx.set_chain_a(saved[3])
    ctx.sweep(2, "measure")
    got = [p.cpu().numpy() for p in ctx.predict()]
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_tiled_and_plain_paths_agree_bitwise():
    zs, gs = ragged_images()
    R = 4
    outs = []
    for path in ("tiled", "plain"):
        ctx = make_ctx(zs, gs, R, path)
        ctx.set_T([0.2, 0.2, 0.1, 0.4])
        ctx.sweep(8, "equil")
        ctx.sweep(4, "measure")
        outs.append(([s.cpu().numpy() for s in ctx.get_state()],
                     [p.cpu().numpy() for p in ctx.predict()]))
    for a, b in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.allclose(a, b, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("tile", [(16, 16), (32, 16), (32, 32)])
def test_tile_shapes_and_chain_groups_agree_bitwise(tile):
    """9 realisations in chain groups of 4 (two groups and a launch of its own for the
    ninth), of 8 (one group and the ninth) and of 9 (one group with a padded row)."""
    zs, gs = ragged_images()
    R = 9
    ref = make_ctx(zs, gs, R, "plain")
    ref.set_T([0.2, 0.2, 0.1, 0.4])
    ref.sweep(3, "equil")
    want = [s.cpu().numpy() for s in ref.get_state()]
    for cg in (4, 8, 9):
        ctx = make_ctx(zs, gs, R, "tiled", tile=tile, chain_group=cg)
        ctx.set_T([0.2, 0.2, 0.1, 0.4])
        ctx.sweep(3, "equil")
        got = [s.cpu().numpy() for s in ctx.get_state()]
        for a, b in zip(got, want):
            assert np.array_equal(a, b)


def _largest_table(gap, tx=16, ty=16):
    """Largest other-colour table of a colour pass over the tiles of one image: the
    gap cells of the other colour inside the tile and in its 1-cell ring (corners
    excluded), plus the zero entry."""
    Ly, Lx = gap.shape
    best = 0
    for y0 in range(0, Ly, ty):
        for x0 in range(0, Lx, tx):
            for c in (0, 1):
                n = 0
                for y in range(max(y0 - 1, 0), min(y0 + ty + 1, Ly)):
                    for x in range(max(x0 - 1, 0), min(x0 + tx + 1, Lx)):
                        corner = not (y0 <= y < y0 + ty) and not (x0 <= x < x0 + tx)
                        if not corner and (x + y) % 2 != c and gap[y, x]:
                            n += 1
                best = max(best, n + 1)
    return best


def test_heavy_tiles_launch_separately_and_agree_bitwise():
    """32 chains in one group: a tile inside the block gap needs a table too large for a
    full SM of blocks and runs in the pass's second (heavy) launch; states, energies
    and sums still equal the plain path's."""
    zs, gs = ragged_images()
    gs[0][16:32, 32:48] = 1  # one 16x16 tile entirely gap
    # 16 pairs x 16 B per entry: more than 92 entries leaves fewer than 8 blocks per SM
    assert _largest_table(gs[0]) > 92
    R = 32
    out = []
    for path, kw in (("plain", {}), ("tiled", {"chain_group": 32})):
        ctx = make_ctx(zs, gs, R, path, **kw)
        ctx.set_T([0.2, 0.2, 0.1, 0.4])
        ctx.sweep(3, "equil", record_energy=True)
        info = ctx.chain_info()
        ctx.sweep(2, "measure")
        out.append(([s.cpu().numpy() for s in ctx.get_state()], info,
                    [p.cpu().numpy() for p in ctx.predict()]))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1]["a"], out[1][1]["a"])
    assert np.array_equal(out[0][1]["accepted"], out[1][1]["accepted"])
    assert np.allclose(out[0][1]["e_last"], out[1][1]["e_last"], rtol=0, atol=1e-6)
    for a, b in zip(out[0][2], out[1][2]):
        assert np.allclose(a, b, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("R,cg", [(32, 32), (36, 16)])
def test_side_stream_launches_in_graphs_equal_the_plain_path(R, cg):
    """With heavy tiles (and, for 36 chains in groups of 16, a launch for the 4 chains
    left over) a colour pass forks its extra launches to a second stream; replayed
    from CUDA graphs on a non-default stream the states, accept counts and a equal
    the plain path's bit for bit."""
    zs, gs = ragged_images()
    gs[0][16:32, 32:48] = 1  # one 16x16 tile entirely gap: a heavy launch
    side = torch.cuda.Stream()
    out = []
    for path, kw in (("plain", {}), ("tiled", {"chain_group": cg})):
        with torch.cuda.stream(side):
            ctx = make_ctx(zs, gs, R, path, **kw)
            ctx.set_T([0.2, 0.2, 0.1, 0.4], stream=side)
            ctx.sweep(6, "equil", stream=side)   # graph replays (runs of 4 or more)
            ctx.sweep(5, "measure", stream=side)
            st = [t.clone() for t in ctx.get_state(stream=side)]
            zh = [t.clone() for t in ctx.predict(stream=side)]
        side.synchronize()
        info = ctx.chain_info()
        out.append(([t.cpu().numpy() for t in st], info, [t.cpu().numpy() for t in zh]))
        ctx.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1]["a"], out[1][1]["a"])
    assert np.array_equal(out[0][1]["accepted"], out[1][1]["accepted"])
    for a, b in zip(out[0][2], out[1][2]):
        assert np.allclose(a, b, rtol=1e-6, atol=1e-5)


def test_determinism_same_state_same_result():
    """Colour-race canary: the same sweep from the same state gives identical bits."""
    zs, gs = ragged_images()
    ctx = make_ctx(zs, gs, 4)
    ctx.set_T([0.2, 0.2, 0.1, 0.4])
    ctx.sweep(2, "equil")
    s0 = [s.clone() for s in ctx.get_state()]
    idx = ctx.sweep_index()
    a0 = ctx.chain_info()["a"]
    ctx.sweep(1, "equil")
    r1 = [s.clone() for s in ctx.get_state()]
    ctx.set_state(s0)
    ctx.set_sweep_index(*idx)
    ctx.set_chain_a(a0)
    ctx.sweep(1, "equil")
    r2 = ctx.get_state()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)


# ------------------------------------------------------------ energy

@pytest.mark.parametrize("path", ["tiled", "plain"])
def test_energy_matches_oracle(path):
    zs, gs = ragged_images()
    ctx = make_ctx(zs, gs, 3, path)
    ctx.set_T([0.2, 0.2, 0.1, 0.4])
    ctx.sweep(5, "equil", record_energy=True)
    e = ctx.energy()
    st = ctx.get_state()
    rec = ctx.chain_info()["e_last"]
    for i in range(len(gs)):
        for c in range(3):
            ref = oracle.specific_energy(st[i][c].cpu().numpy().astype(np.float64))
            assert abs(e[i, c] - ref) < 1e-6
            assert abs(rec[i, c] - ref) < 2e-6


def test_energy_autograd_matches_finite_differences_and_oracle():
    rng = np.random.default_rng(3)
    phi_np = rng.uniform(0, TWO_PI, (2, 24, 31))
    phi = torch.tensor(phi_np, dtype=torch.float32, device="cuda", requires_grad=True)
    J = torch.tensor(1.3, dtype=torch.float64, requires_grad=True)
    H = mpr.MPREnergy.apply(phi, J)
    w = torch.tensor([0.7, -1.1], dtype=torch.float64, device="cuda")
    (H * w).sum().backward()
    for k in range(2):
        p64 = phi.detach()[k].cpu().numpy().astype(np.float64)
        assert abs(H[k].item() - oracle.energy(p64, J=1.3)) < 1e-4 * abs(H[k].item()) + 1e-4
        g_ref = oracle.torque(p64, J=1.3) * w[k].item()
        assert np.max(np.abs(phi.grad[k].cpu().numpy() - g_ref)) < 1e-5
        # central differences (h = 1e-3, FP64) on a few sites
        for (y, x) in [(0, 0), (5, 7), (23, 30), (12, 0)]:
            a = p64.copy(); a[y, x] += 1e-3
            b = p64.copy(); b[y, x] -= 1e-3
            fd = (oracle.energy(a, J=1.3) - oracle.energy(b, J=1.3)) / 2e-3 * w[k].item()
            assert abs(phi.grad[k, y, x].item() - fd) < 1e-5
    # dH/dJ = H / J = -sum cos(q dphi), the energy at J = 1
    dJ = sum(w[k].item() * oracle.energy(phi.detach()[k].cpu().numpy().astype(np.float64), J=1.0)
             for k in range(2))
    assert abs(J.grad.item() - dJ) < 1e-4 * abs(dJ) + 1e-4


# ------------------------------------------------ long runs, statistics

def test_long_run_statistics_and_prediction_grf64():
    """Config 1 (64 x 64 GRF, 33% gaps, 10 chains, 200 + 100 sweeps) at fixed T:
    mean specific energy within 3 sigma and MAE/RMSE within 2% of the oracle."""
    w = synthetic.workload("grf64")
    z, g = w.z[0], w.gap[0]
    T = 0.13
    R, ne, nm = w.chains, w.n_equil, w.n_meas
    ctx = make_ctx([z], [g], R)
    ctx.set_T([T])
    ctx.sweep(ne, "equil")
    es = []
    for _ in range(nm):
        ctx.sweep(1, "measure", record_energy=True)
        es.append(ctx.chain_info()["e_last"][0])
    es = np.array(es)                      # [nm, R]
    zh = ctx.predict()[0].cpu().numpy()
    phi, zmin, zmax = oracle.map_to_angles(z.astype(np.float64), g)
    sim = oracle.simulate(phi, g, T=T, R=R, n_equil=ne, n_meas=nm, seed=SEED + 1, history=True)
    e_or = sim["e_hist"][:, ne:]           # [R, nm]
    # chains are independent: sigma from the spread of chain means
    m_g, m_o = es.mean(0), e_or.mean(1)
    sig = math.sqrt(m_g.var(ddof=1) / R + m_o.var(ddof=1) / R)
    assert abs(m_g.mean() - m_o.mean()) < 3 * sig + 1e-6, (m_g.mean(), m_o.mean(), sig)
    zo = oracle.unmap(sim["phi_mean"], zmin, zmax)
    truth = z.astype(np.float64)
    m = g == 1
    mae_g, mae_o = np.mean(np.abs(zh[m] - truth[m])), np.mean(np.abs(zo[m] - truth[m]))
    rmse_g = math.sqrt(np.mean((zh[m] - truth[m]) ** 2))
    rmse_o = math.sqrt(np.mean((zo[m] - truth[m]) ** 2))
    assert abs(mae_g - mae_o) < 0.02 * mae_o, (mae_g, mae_o)
    assert abs(rmse_g - rmse_o) < 0.02 * rmse_o, (rmse_g, rmse_o)
    # sample pixels are returned unchanged
    assert np.array_equal(zh[~m], z[~m])


def test_long_run_statistics_lognormal256(golden_dir):
    """A 256 x 256 field shaped like the 1024 x 1024 lognormal workload (Matern
    nu = 1.5, ell = 20, log-std 0.8, 50% gaps), 100 realisations: the SEM temperature
    within 1% of the oracle's bisection, and at the oracle's T the mean specific
    energy within 3 sigma and MAE / RMSE within 2% of the oracle's long run (the
    oracle's figures from tests/golden/make_longrun_lognormal256.py)."""
    import json
    with open(os.path.join(golden_dir, "lognormal256_longrun.json")) as f:
        ref = json.load(f)
    w = synthetic.workload("lognormal1024", L=ref["input"]["side"])
    z, g = w.z[0], w.gap[0]
    sim = ref["simulate"]
    R = sim["blocks"] * sim["chains_per_block"]
    ne, nm = sim["n_equil"], sim["n_meas"]
    sem = ref["sem"]
    topts = mpr.TOpts(L=sem["L"], chains=16, n_equil=60, n_meas=120, iters=6)
    ctx = mpr.Context([z], [g], chains=R, params=mpr.Params(seed=SEED + 7), topts=topts)
    assert abs(ctx.image_info()["e_s"][0] - ref["e_s"]) < 1e-6
    T_gpu = ctx.estimate_T()[0]
    assert abs(T_gpu - sem["T"]) < 0.01 * sem["T"], (T_gpu, sem["T"])
    ctx.set_T([sem["T"]])
    ctx.sweep(ne, "equil")
    es = []
    for _ in range(nm):
        ctx.sweep(1, "measure", record_energy=True)
        es.append(ctx.chain_info()["e_last"][0])
    m_g = np.array(es).mean(0)              # per-realisation means
    m_o = np.array(ref["e_chain_mean"])
    sig = math.sqrt(m_g.var(ddof=1) / len(m_g) + m_o.var(ddof=1) / len(m_o))
    # at this T the chains' energies spread by a few 1e-7 only, the size of the FP32
    # energy evaluation's own error: that error, measured on the final states (the
    # recorded FP32 energy against the FP64 energy of the same angles), is allowed
    # on top of 3 sigma
    fin = ctx.get_state()[0].cpu().numpy().astype(np.float64)
    e_fp64 = np.array([oracle.specific_energy(fin[c]) for c in range(R)])
    bias = float(np.mean(np.array(es[-1]) - e_fp64))
    assert abs(bias) < 2e-6
    assert abs(m_g.mean() - m_o.mean()) < 3 * sig + abs(bias), (m_g.mean(), m_o.mean(), sig, bias)
    zh = ctx.predict()[0].cpu().numpy().astype(np.float64)
    m = g == 1
    err = zh[m] - z[m].astype(np.float64)
    mae, rmse = float(np.mean(np.abs(err))), float(np.sqrt(np.mean(err ** 2)))
    assert abs(mae - ref["mae"]) < 0.02 * ref["mae"], (mae, ref["mae"])
    assert abs(rmse - ref["rmse"]) < 0.02 * ref["rmse"], (rmse, ref["rmse"])
    ctx.close()


def test_estimate_T_newton_matches_oracle_bisection():
    """SEM temperature: GPU Newton (fluctuation relation) vs oracle bisection within 1%."""
    w = synthetic.workload("grf64")
    z, g = w.z[0], w.gap[0]
    topts = mpr.TOpts(L=64, chains=4, n_equil=60, n_meas=120, iters=6)
    ctx = mpr.Context([z], [g], chains=2, params=mpr.Params(seed=SEED), topts=topts)
    T_gpu = ctx.estimate_T()[0]
    e_s = ctx.image_info()["e_s"][0]
    T_or = oracle.estimate_T(e_s, L=64, K=2, n_eq=120, n_meas=120, seed=SEED, rel_tol=2e-3)
    assert abs(T_gpu - T_or) < 0.01 * T_or, (T_gpu, T_or)


# ------------------------------------------------------------ errors

def test_host_errors():
    z = np.full((8, 8), 3.0, np.float32)
    g = np.zeros((8, 8), np.uint8)
    g[0, 0] = 1
    with pytest.raises(mpr._lib.MprError) as e:
        mpr.Context([z], [g], chains=2)
    assert e.value.status == 3  # degenerate range
    z2 = np.arange(64, dtype=np.float32).reshape(8, 8)
    cb = np.fromfunction(lambda y, x: (x + y) % 2, (8, 8)).astype(np.uint8)
    ctx = mpr.Context([z2], [cb], chains=2)
    with pytest.raises(mpr._lib.MprError) as e:
        ctx.estimate_T()
    assert e.value.status == 4  # no sample pairs
    with pytest.raises(mpr._lib.MprError) as e:
        ctx.sweep(1)
    assert e.value.status == 7  # T not set
    with pytest.raises(mpr._lib.MprError):
        ctx.predict()


def _tiny_images():
    """Degenerate shapes: 2x2 with one gap, single-row and single-column-pair
    images, 3x3, and a nearly empty image (two samples left)."""
    rng = np.random.default_rng(9)
    out = []
    for (h, w, frac) in ((2, 2, 0.25), (2, 9, 0.5), (9, 2, 0.5), (3, 3, 0.6), (7, 11, 0.95)):
        z = rng.normal(50, 10, (h, w)).astype(np.float32)
        g = synthetic.uniform_gaps((h, w), frac, int(rng.integers(1 << 30))).astype(np.uint8)
        if (g == 0).sum() < 2:  # keep at least two samples
            g.ravel()[:2] = 0
        out.append((z, g))
    return [o[0] for o in out], [o[1] for o in out]


@pytest.mark.parametrize("path", ["tiled", "plain"])
def test_degenerate_shapes_sweep_parity(path):
    zs, gs = _tiny_images()
    R = 3
    ctx = make_ctx(zs, gs, R, path)
    T = np.array([0.3, 0.2, 0.25, 0.15, 0.4])
    ctx.set_T(T)
    ctx.sweep(2, "equil")
    tally = Tally()
    for _ in range(3):
        before = [s.cpu().numpy() for s in ctx.get_state()]
        a = ctx.chain_info()["a"]
        s_idx, _ = ctx.sweep_index()
        ctx.sweep(1, "equil", record_energy=True)
        after = [s.cpu().numpy() for s in ctx.get_state()]
        info = ctx.chain_info()
        for i, g in enumerate(gs):
            for c in range(R):
                compare_sweep(before[i][c], after[i][c], g, tally, T=T[i], a=a[i, c], seed=SEED,
                              img=i, chain=c, sweep_index=s_idx)
                e_ref = oracle.specific_energy(after[i][c].astype(np.float64))
                assert abs(info["e_last"][i, c] - e_ref) < 2e-6
    tally.assert_budget()
    ctx.sweep(4, "measure")
    for z, g, p in zip(zs, gs, ctx.predict()):
        p = p.cpu().numpy()
        assert np.array_equal(p[g == 0], z[g == 0])
        assert np.all(np.isfinite(p))


@pytest.mark.parametrize("path", ["tiled", "plain"])
def test_longest_sides_sweep_parity(path):
    """Images at the longest side the layout allows (65535: the random stream's
    counter keeps y in 16 bits and x >> 1 in 16), as 2-row and 2-column strips:
    two sweeps against the oracle under the decision-parity rule."""
    shapes = [(2, 65535), (65535, 2)]
    zs, gs = [], []
    for k, (h, w) in enumerate(shapes):
        rng = np.random.default_rng(70 + k)
        zs.append((50 + 10 * np.cumsum(rng.standard_normal(h * w)) / 100).reshape(h, w).astype(np.float32))
        gs.append(synthetic.uniform_gaps((h, w), 0.4, 80 + k).astype(np.uint8))
    R = 2
    ctx = make_ctx(zs, gs, R, path)
    T = np.array([0.2, 0.3])
    ctx.set_T(T)
    n_main, n_T = ctx.sweep_launches()
    assert n_main >= 3 and n_T >= 3
    tally = Tally()
    for _ in range(2):
        before = [s.cpu().numpy() for s in ctx.get_state()]
        a = ctx.chain_info()["a"]
        s_idx, _ = ctx.sweep_index()
        ctx.sweep(1, "equil")
        after = [s.cpu().numpy() for s in ctx.get_state()]
        for i, g in enumerate(gs):
            for c in range(R):
                compare_sweep(before[i][c], after[i][c], g, tally, T=T[i], a=a[i, c], seed=SEED,
                              img=i, chain=c, sweep_index=s_idx)
    tally.assert_budget()
    print(tally)
