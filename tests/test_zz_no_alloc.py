"""The allocation-free entry point against the context's own sample energy.

mpr_sample_energy_noalloc() serves callers that may not allocate device
memory (its scratch is a fixed array inside the library).  It must report
what mpr_init_grid() computes for the same images, on every call: its
scratch keeps the previous call's contents, so two calls in a row are
compared.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1710_03038_gb300 as mpr  # noqa: E402
from paper_1710_03038_gb300 import _lib  # noqa: E402


def _images():
    shapes = [(64, 64), (37, 53), (130, 5), (300, 211)]
    zs, gs = [], []
    for k, (h, w) in enumerate(shapes):
        z = synthetic.grf((h, w), nu=0.5, ell=5.0 + 3 * k, mean=50, std=10, seed=300 + k)
        g = synthetic.uniform_gaps((h, w), 0.2 + 0.15 * k, 400 + k)
        zs.append(torch.from_numpy(z.astype(np.float32)).cuda())
        gs.append(torch.from_numpy(g.astype(np.uint8)).cuda())
    return zs, gs


def test_noalloc_sample_energy_matches_init_grid_twice():
    zs, gs = _images()
    ref = mpr.Context(zs, gs, chains=1).image_info()
    n = len(zs)
    out = dict(e_s=torch.empty(n, dtype=torch.float64, device="cuda"),
               n_sp=torch.empty(n, dtype=torch.int64, device="cuda"),
               zmin=torch.empty(n, dtype=torch.float32, device="cuda"),
               zmax=torch.empty(n, dtype=torch.float32, device="cuda"))
    for _ in range(2):
        for v in out.values():
            v.fill_(-7)  # stale values must be overwritten
        got = mpr.sample_energy_noalloc(zs, gs, out=out)
        torch.cuda.synchronize()
        e = got["e_s"].cpu().numpy()
        assert np.allclose(e, ref["e_s"], rtol=1e-12, atol=1e-14), (e, ref["e_s"])
        assert np.array_equal(got["n_sp"].cpu().numpy(), ref["n_sp"])
        assert np.array_equal(got["zmin"].cpu().numpy(), ref["zmin"])
        assert np.array_equal(got["zmax"].cpu().numpy(), ref["zmax"])


def test_noalloc_concatenated_inputs_and_degenerate_images():
    """The concatenated form (nothing allocated by the wrapper) on images without a
    usable sample energy: constant sample values (z_max = z_min) and a checkerboard
    mask (no sample pair) give e_s = nan and N_SP = 0; a regular image next to them
    is unaffected."""
    zc = torch.full((8, 8), 3.0, dtype=torch.float32, device="cuda")
    gc = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    gc[0, 0] = 1
    zk = torch.arange(64, dtype=torch.float32, device="cuda").reshape(8, 8)
    yy, xx = torch.meshgrid(torch.arange(8), torch.arange(8), indexing="ij")
    gk = ((xx + yy) % 2).to(torch.uint8).cuda()
    zs, gs = _images()
    zs, gs = [zc, zk, zs[0]], [gc, gk, gs[0]]
    shapes = [tuple(t.shape) for t in gs]
    zf = torch.cat([t.reshape(-1) for t in zs]).contiguous()
    gf = torch.cat([t.reshape(-1) for t in gs]).contiguous()
    n = len(zs)
    out = dict(e_s=torch.empty(n, dtype=torch.float64, device="cuda"),
               n_sp=torch.empty(n, dtype=torch.int64, device="cuda"),
               zmin=torch.empty(n, dtype=torch.float32, device="cuda"),
               zmax=torch.empty(n, dtype=torch.float32, device="cuda"))
    for _ in range(2):
        got = mpr.sample_energy_noalloc(zf, gf, out=out, shapes=shapes)
        torch.cuda.synchronize()
        e = got["e_s"].cpu().numpy()
        nsp = got["n_sp"].cpu().numpy()
        assert np.isnan(e[0]) and nsp[0] == 0
        assert np.isnan(e[1]) and nsp[1] == 0
        ref = mpr.Context([zs[2]], [gs[2]], chains=1).image_info()
        assert np.allclose(e[2], ref["e_s"][0], rtol=1e-12, atol=1e-14)
        assert nsp[2] == ref["n_sp"][0]


def test_noalloc_rejects_more_images_than_its_scratch_holds():
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    g = torch.zeros(4, dtype=torch.uint8, device="cuda")
    n = 65
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    import ctypes as C
    lib = _lib.load()
    st = lib.mpr_sample_energy_noalloc(n, _lib.int_array([2] * n), _lib.int_array([2] * n),
                                       C.c_void_p(z.data_ptr()), C.c_void_p(g.data_ptr()),
                                       0.5, 1.0, C.c_void_p(e.data_ptr()), None, None, None, None)
    assert st == 1
    assert b"64" in lib.mpr_last_error()
