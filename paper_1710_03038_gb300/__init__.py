"""GB300-native gap filling with the modified planar rotator (MPR) Gibbs random field.

Thin Python layer over the C ABI of ``include/mpr.h``: it owns device memory
(torch tensors) and streams and marshals arguments; every step of the method
runs in the library's CUDA kernels.

    ctx = Context([z], [gap], chains=32)      # Alg. 2 steps 1-3.1
    ctx.estimate_T()                           # Sec. 2.3, specific energy matching
    ctx.sweep(50, "equil")                     # Alg. 2 step 4
    ctx.sweep(100, "measure")                  # Alg. 2 step 5
    z_hat = ctx.predict()                      # conditional mean
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from ._lib import MprParams, MprTOpts, call, int_array, i64_array

__all__ = ["Params", "TOpts", "Context", "fill", "MPREnergy", "lattice_energy", "lattice_torque",
           "lattice_grad", "philox", "version", "workspace_size", "eT_table", "select_q",
           "autotune", "sample_energy_noalloc"]


def version() -> str:
    return _lib.load().mpr_version().decode()


@dataclass
class Params:
    """Model and simulation parameters (defaults: the paper's values)."""
    q: float = 0.5
    J: float = 1.0
    A_targ: float = 0.3
    k_a: float = 3.0
    seed: int = 0x2545F4914F6CDD1D
    freeze_a_in_measure: bool = True
    path: str = "tiled"          # "tiled" (batched) or "plain"
    tile: tuple = (0, 0)         # (tile_x, tile_y); (0, 0) = 16x16
    chain_group: int = 0         # chains per thread block (multiple of 4); 0 = automatic
    literal_or: bool = False     # printed q = 1 over-relaxation (comparison only)
    use_graphs: bool = True      # replay captured CUDA graphs of sweep runs (non-default streams)
    model: str = "mpr"           # "mpr" or "gmrf" (Sec. 4.3 pair interaction)

    def c(self) -> MprParams:
        p = MprParams()
        call("mpr_default_params", C.byref(p))
        p.q, p.J, p.A_targ, p.k_a = self.q, self.J, self.A_targ, self.k_a
        p.seed = int(self.seed) & ((1 << 64) - 1)
        p.freeze_a_in_measure = int(bool(self.freeze_a_in_measure))
        p.path = {"tiled": _lib.MPR_PATH_TILED, "plain": _lib.MPR_PATH_PLAIN}[self.path]
        p.tile_x, p.tile_y = int(self.tile[0]), int(self.tile[1])
        p.chain_group = int(self.chain_group)
        p.literal_or = int(bool(self.literal_or))
        p.use_graphs = int(bool(self.use_graphs))
        p.model = {"mpr": _lib.MPR_MODEL_MPR, "gmrf": _lib.MPR_MODEL_GMRF}[self.model]
        return p


@dataclass
class TOpts:
    """Options of the temperature estimate (unconditional lattice side, chains, sweeps)."""
    L: int = 0
    chains: int = 16
    n_equil: int = 40
    n_meas: int = 40
    iters: int = 4
    T_lo: float = 1e-5
    T_hi: float = 20.0

    def c(self) -> MprTOpts:
        o = MprTOpts()
        o.L, o.chains, o.n_equil, o.n_meas, o.iters = (int(self.L), int(self.chains),
                                                       int(self.n_equil), int(self.n_meas),
                                                       int(self.iters))
        o.T_lo, o.T_hi = float(self.T_lo), float(self.T_hi)
        return o


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _as_list(x):
    if isinstance(x, (list, tuple)):
        return list(x)
    if isinstance(x, torch.Tensor) and x.dim() == 2:
        return [x]
    if isinstance(x, np.ndarray) and x.ndim == 2:
        return [x]
    return list(x)


def workspace_size(shapes, n_gap, chains, params: Params = None, topts: TOpts = None) -> int:
    params = params or Params()
    topts = topts or TOpts()
    n = len(shapes)
    Ly = int_array([s[0] for s in shapes])
    Lx = int_array([s[1] for s in shapes])
    ng = i64_array(n_gap) if n_gap is not None else None
    out = C.c_size_t()
    call("mpr_workspace_size", n, Lx, Ly, ng, int(chains), C.byref(params.c()),
         C.byref(topts.c()), C.byref(out))
    return out.value


class Context:
    """A batch of gappy images and their realisations on one GPU (an mpr_ctx).

    z, gap: sequences of 2-D arrays (numpy, or torch tensors on the host or on
    the current CUDA device); gap nonzero = missing.  Inputs on the host are
    copied by the library (``where="host"``), device tensors are read in
    place.
    """

    def __init__(self, z, gap, chains: int, params: Params = None, topts: TOpts = None,
                 device=None, stream=None):
        self.params = params or Params()
        self.topts = topts or TOpts()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        zs = _as_list(z)
        gs = _as_list(gap)
        if len(zs) != len(gs):
            raise ValueError("z and gap must have the same number of images")
        self.shapes = [tuple(int(v) for v in g.shape) for g in gs]
        self.n_img = len(self.shapes)
        self.chains = int(chains)
        on_dev = isinstance(zs[0], torch.Tensor) and zs[0].is_cuda
        if on_dev:
            zf = torch.cat([t.reshape(-1).to(torch.float32) for t in zs]).contiguous()
            gf = torch.cat([(t.reshape(-1) != 0).to(torch.uint8) for t in gs]).contiguous()
            where = _lib.MPR_DEVICE
            ng = [int(g.count_nonzero()) for g in gs]
        elif (len(zs) == 1 and isinstance(zs[0], torch.Tensor) and isinstance(gs[0], torch.Tensor)
              and zs[0].dtype == torch.float32 and gs[0].dtype in (torch.uint8, torch.bool)
              and zs[0].is_contiguous() and gs[0].is_contiguous()
              and zs[0].is_pinned() and gs[0].is_pinned()):
            # pinned host buffers of the library's types: handed over as they are
            zf = zs[0].reshape(-1)
            gf = gs[0].reshape(-1).view(torch.uint8)
            where = _lib.MPR_HOST
            # no host pass over the mask: the workspace is sized for the worst case
            # (every site a gap) and the library counts the gaps on the device
            ng = None
        else:
            zn = [np.asarray(t.cpu() if isinstance(t, torch.Tensor) else t, dtype=np.float32) for t in zs]
            gn = [(np.asarray(t.cpu() if isinstance(t, torch.Tensor) else t) != 0).astype(np.uint8) for t in gs]
            zf = torch.from_numpy(np.concatenate([a.ravel() for a in zn])).pin_memory()
            gf = torch.from_numpy(np.concatenate([a.ravel() for a in gn])).pin_memory()
            where = _lib.MPR_HOST
            ng = [int(a.sum()) for a in gn]
        self.n_sites = int(sum(a * b for a, b in self.shapes))
        Ly = int_array([s[0] for s in self.shapes])
        Lx = int_array([s[1] for s in self.shapes])
        cp, co = self.params.c(), self.topts.c()
        nbytes = C.c_size_t()
        call("mpr_workspace_size", self.n_img, Lx, Ly, i64_array(ng) if ng is not None else None,
             self.chains, C.byref(cp),
             C.byref(co), C.byref(nbytes))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self._ctx = C.c_void_p()
        call("mpr_init_grid", C.byref(self._ctx), self.n_img, Lx, Ly, self.chains, C.byref(cp),
             C.byref(co), _ptr(zf), _ptr(gf), where, _ptr(self.workspace),
             C.c_size_t(self.workspace.numel()), _stream_ptr(stream))
        self._inputs = (zf, gf)

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            _lib.load().mpr_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- info --------------------------------------------------------------
    def image_info(self) -> dict:
        n = self.n_img
        e_s = (C.c_double * n)()
        nsp = (C.c_int64 * n)()
        ngap = (C.c_int64 * n)()
        zmin = (C.c_float * n)()
        zmax = (C.c_float * n)()
        call("mpr_get_image_info", self._ctx, e_s, nsp, ngap, zmin, zmax)
        return dict(e_s=np.array(e_s[:]), n_sp=np.array(nsp[:]), n_gap=np.array(ngap[:]),
                    zmin=np.array(zmin[:]), zmax=np.array(zmax[:]))

    # -- temperature -----------------------------------------------------------
    def estimate_T(self, stream=None) -> np.ndarray:
        T = (C.c_double * self.n_img)()
        call("mpr_estimate_T", self._ctx, T, _stream_ptr(stream))
        return np.array(T[:])

    def estimate_T_async(self, stream=None):
        call("mpr_estimate_T", self._ctx, None, _stream_ptr(stream))

    def set_T_from_table(self, T_grid, e_grid, stream=None) -> np.ndarray:
        """T_hat = e^-1(e_s) from an e(T) table (see eT_table); returns T per image."""
        n = len(T_grid)
        Tg = (C.c_double * n)(*[float(v) for v in T_grid])
        eg = (C.c_double * n)(*[float(v) for v in e_grid])
        out = (C.c_double * self.n_img)()
        call("mpr_set_T_from_table", self._ctx, n, Tg, eg, out, _stream_ptr(stream))
        return np.array(out[:])

    def set_T(self, T, stream=None):
        T = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_img,))
        call("mpr_set_T", self._ctx, (C.c_double * self.n_img)(*T), _stream_ptr(stream))

    def get_T(self, stream=None) -> np.ndarray:
        T = (C.c_double * self.n_img)()
        call("mpr_get_T", self._ctx, T, _stream_ptr(stream))
        return np.array(T[:])

    # -- sweeps ----------------------------------------------------------------
    def sweep(self, n: int, phase: str = "equil", record_energy: bool = False, stream=None):
        ph = {"equil": _lib.MPR_EQUIL, "measure": _lib.MPR_MEASURE}[phase]
        call("mpr_sweep", self._ctx, int(n), ph, _lib.MPR_RECORD_ENERGY if record_energy else 0,
             _stream_ptr(stream))

    def equilibrate(self, n_f: int = 5, n_fit: int = 20, i_max: int = 500, stream=None) -> int:
        """Equilibrate until the degree-1 Savitzky-Golay slope of every image's
        chain-mean energy is no longer negative (Alg. 2 step 4); returns sweeps run."""
        n = C.c_int()
        call("mpr_equilibrate", self._ctx, int(n_f), int(n_fit), int(i_max), C.byref(n),
             _stream_ptr(stream))
        return n.value

    def energy_history(self, stream=None) -> np.ndarray:
        """[n_img, 512] ring of chain-mean energies of the last equilibrate() (entry i % 512)."""
        out = (C.c_double * (self.n_img * 512))()
        call("mpr_get_energy_history", self._ctx, out, _stream_ptr(stream))
        return np.array(out[:]).reshape(self.n_img, 512)

    def energy(self, stream=None) -> np.ndarray:
        out = (C.c_double * (self.n_img * self.chains))()
        call("mpr_energy", self._ctx, C.cast(out, C.c_void_p), _lib.MPR_HOST, _stream_ptr(stream))
        return np.array(out[:]).reshape(self.n_img, self.chains)

    def predict(self, std: bool = False, stream=None):
        """Conditional mean (and std) per image as device tensors."""
        zh = torch.empty(self.n_sites, dtype=torch.float32, device=self.device)
        zs = torch.empty(self.n_sites, dtype=torch.float32, device=self.device) if std else None
        call("mpr_predict", self._ctx, _ptr(zh), _ptr(zs) if std else None, _lib.MPR_DEVICE,
             _stream_ptr(stream))
        out = self._split(zh)
        return (out, self._split(zs)) if std else out

    def predict_host(self, out: torch.Tensor, std_out: torch.Tensor = None, stream=None):
        """Conditional mean into a (pinned) host buffer of n_sites floats; blocking."""
        call("mpr_predict", self._ctx, _ptr(out), _ptr(std_out) if std_out is not None else None,
             _lib.MPR_HOST, _stream_ptr(stream))

    def reset_accumulators(self, stream=None):
        call("mpr_reset_accumulators", self._ctx, _stream_ptr(stream))

    def accumulators(self, stream=None):
        """Realisation sums of phi and phi^2 per gap pixel (lists per image of [Ly, Lx]
        float64 device tensors, 0 at samples) and their number of terms."""
        s1 = torch.empty(self.n_sites, dtype=torch.float64, device=self.device)
        s2 = torch.empty(self.n_sites, dtype=torch.float64, device=self.device)
        n = C.c_int64()
        call("mpr_get_accumulators", self._ctx, _ptr(s1), _ptr(s2), C.byref(n), _lib.MPR_DEVICE,
             _stream_ptr(stream))
        return self._split(s1), self._split(s2), n.value

    def set_accumulators(self, sums, sums2, n_terms: int, stream=None):
        """Restore realisation sums (as returned by accumulators()); sums2 may be None."""
        s1 = torch.cat([torch.as_tensor(t, dtype=torch.float64, device=self.device).reshape(-1)
                        for t in _as_list(sums)]).contiguous()
        s2 = None
        if sums2 is not None:
            s2 = torch.cat([torch.as_tensor(t, dtype=torch.float64, device=self.device).reshape(-1)
                            for t in _as_list(sums2)]).contiguous()
        call("mpr_set_accumulators", self._ctx, _ptr(s1), _ptr(s2) if s2 is not None else None,
             C.c_int64(int(n_terms)), _lib.MPR_DEVICE, _stream_ptr(stream))
        self._keep = (s1, s2)

    def _split(self, flat):
        out, off = [], 0
        for (h, w) in self.shapes:
            out.append(flat[off:off + h * w].view(h, w))
            off += h * w
        return out

    # -- state -------------------------------------------------------------------
    def get_state(self, stream=None):
        """Angles of every realisation: list per image of [chains, Ly, Lx] device tensors."""
        flat = torch.empty(self.n_sites * self.chains, dtype=torch.float32, device=self.device)
        call("mpr_get_state", self._ctx, _ptr(flat), _lib.MPR_DEVICE, _stream_ptr(stream))
        out, off = [], 0
        for (h, w) in self.shapes:
            n = h * w * self.chains
            out.append(flat[off:off + n].view(self.chains, h, w))
            off += n
        return out

    def set_state(self, states, stream=None):
        flat = torch.cat([torch.as_tensor(s, dtype=torch.float32, device=self.device).reshape(-1)
                          for s in _as_list(states)]).contiguous()
        if flat.numel() != self.n_sites * self.chains:
            raise ValueError("state has the wrong size")
        call("mpr_set_state", self._ctx, _ptr(flat), _lib.MPR_DEVICE, _stream_ptr(stream))
        torch.cuda.current_stream().synchronize()

    def chain_info(self, stream=None) -> dict:
        n = self.n_img * self.chains
        a = (C.c_float * n)()
        acc = (C.c_uint32 * n)()
        e = (C.c_double * n)()
        call("mpr_get_chain_info", self._ctx, a, acc, e, _stream_ptr(stream))
        shp = (self.n_img, self.chains)
        return dict(a=np.array(a[:]).reshape(shp), accepted=np.array(acc[:]).reshape(shp),
                    e_last=np.array(e[:]).reshape(shp))

    def set_chain_a(self, a, stream=None):
        a = np.asarray(a, dtype=np.float32).reshape(-1)
        a = np.broadcast_to(a, (self.n_img * self.chains,)).copy()
        call("mpr_set_chain_a", self._ctx, a.ctypes.data_as(C.POINTER(C.c_float)), _stream_ptr(stream))

    def sweep_index(self):
        s, e = C.c_uint32(), C.c_uint32()
        call("mpr_get_sweep_index", self._ctx, C.byref(s), C.byref(e))
        return s.value, e.value

    def sweep_launches(self):
        """Kernel launches per sweep of the realisations and of the temperature lattices."""
        m, t = C.c_int(), C.c_int()
        call("mpr_sweep_launches", self._ctx, C.byref(m), C.byref(t))
        return m.value, t.value

    def set_sweep_index(self, sweep: int, equil_index: int, stream=None):
        call("mpr_set_sweep_index", self._ctx, C.c_uint32(sweep), C.c_uint32(equil_index),
             _stream_ptr(stream))


def autotune(z, gap, chains: int, params: Params = None, sweeps: int = 3, device=None, stream=None):
    """Time the tiled path's tile shapes and chain groups on this batch; returns
    (tuned Params, {(tile, chain_group): ms per sweep})."""
    import dataclasses
    params = params or Params()
    zs, gs = _as_list(z), _as_list(gap)
    shapes = [tuple(int(v) for v in g.shape) for g in gs]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    zf = torch.cat([torch.as_tensor(t, device=dev).reshape(-1).to(torch.float32) for t in zs]).contiguous()
    gf = torch.cat([(torch.as_tensor(t, device=dev).reshape(-1) != 0).to(torch.uint8) for t in gs]).contiguous()
    probe = dataclasses.replace(params, tile=(16, 16))
    nbytes = workspace_size(shapes, None, chains, probe)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    p = params.c()
    t = (C.c_double * 9)()
    call("mpr_autotune", len(shapes), int_array([s[1] for s in shapes]),
         int_array([s[0] for s in shapes]), int(chains), C.byref(p), _ptr(zf), _ptr(gf),
         _lib.MPR_DEVICE, _ptr(ws), C.c_size_t(ws.numel()), int(sweeps), t, _stream_ptr(stream))
    tiles = [(32, 16), (16, 16), (32, 32)]
    groups = [0, 8, 2]
    times = {(tiles[i // 3], groups[i % 3]): t[i] for i in range(9) if t[i] >= 0}
    return dataclasses.replace(params, tile=(p.tile_x, p.tile_y), chain_group=p.chain_group), times


def eT_table(T_grid, L: int = 256, chains: int = 16, n_equil: int = 60, n_meas: int = 60,
             params: Params = None, device=None, stream=None):
    """e(T, L) on unconditional L x L lattices at every T of T_grid -> (e, Var(e)) arrays."""
    params = params or Params()
    n = len(T_grid)
    nbytes = C.c_size_t()
    call("mpr_eT_table_workspace_size", int(L), n, int(chains), C.byref(nbytes))
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
    Tg = (C.c_double * n)(*[float(v) for v in T_grid])
    e = (C.c_double * n)()
    v = (C.c_double * n)()
    call("mpr_eT_table", int(L), n, Tg, int(chains), int(n_equil), int(n_meas),
         C.byref(params.c()), _ptr(ws), C.c_size_t(ws.numel()), e, v, _stream_ptr(stream))
    return np.array(e[:]), np.array(v[:])


def select_q(z, gap, holdout, qs, chains: int = 16, n_equil: int = 100, n_meas: int = 100,
             params: Params = None, topts: TOpts = None, device=None, stream=None):
    """Cross-validated q (mpr_select_q): the samples flagged in `holdout` are the
    validation set; every candidate q runs the gap fill and is scored by the mean
    absolute error at the validation points -> dict(q, scores, T)."""
    params = params or Params()
    topts = topts or TOpts()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    zt = torch.as_tensor(np.asarray(z) if not torch.is_tensor(z) else z).to(dev, torch.float32).contiguous()
    gt = torch.as_tensor(np.asarray(gap) if not torch.is_tensor(gap) else gap).to(dev, torch.uint8).contiguous()
    ht = torch.as_tensor(np.asarray(holdout) if not torch.is_tensor(holdout) else holdout)
    ht = ht.to(dev, torch.uint8).contiguous()
    Ly, Lx = zt.shape
    if tuple(gt.shape) != (Ly, Lx) or tuple(ht.shape) != (Ly, Lx):
        raise ValueError("z, gap and holdout must have one shape")
    pc, tc = params.c(), topts.c()
    nbytes = C.c_size_t()
    call("mpr_select_q_workspace_size", int(Lx), int(Ly), int(chains), C.byref(pc), C.byref(tc),
         C.byref(nbytes))
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
    n = len(qs)
    qa = (C.c_double * n)(*[float(v) for v in qs])
    sc = (C.c_double * n)()
    Ts = (C.c_double * n)()
    qb = C.c_double()
    call("mpr_select_q", int(Lx), int(Ly), _ptr(zt), _ptr(gt), _ptr(ht), _lib.MPR_DEVICE, n, qa,
         int(chains), int(n_equil), int(n_meas), C.byref(pc), C.byref(tc), _ptr(ws),
         C.c_size_t(ws.numel()), sc, Ts, C.byref(qb), _stream_ptr(stream))
    return dict(q=qb.value, scores=np.array(sc[:]), T=np.array(Ts[:]))


def fill(z, gap, chains: int, n_equil: int, n_meas: int, params: Params = None,
         topts: TOpts = None, T=None, std: bool = False):
    """Whole gap fill (Alg. 2): init, SEM temperature (unless T given), sweeps, prediction."""
    ctx = Context(z, gap, chains, params, topts)
    if T is None:
        ctx.estimate_T_async()
    else:
        ctx.set_T(T)
    ctx.sweep(n_equil, "equil")
    ctx.sweep(n_meas, "measure")
    out = ctx.predict(std=std)
    return out, ctx


# ---------------------------------------------------------------- energy autograd

def lattice_energy(phi: torch.Tensor, q: float = 0.5, J: float = 1.0, stream=None) -> torch.Tensor:
    """H (FP64) of a [..., Ly, Lx] float32 CUDA tensor of angles, one value per leading index."""
    Ly, Lx = phi.shape[-2:]
    n = int(np.prod(phi.shape[:-2])) if phi.dim() > 2 else 1
    p = phi.contiguous()
    H = torch.empty(n, dtype=torch.float64, device=phi.device)
    call("mpr_lattice_energy", n, int_array([Lx] * n), int_array([Ly] * n), _ptr(p), float(q),
         float(J), _ptr(H), _stream_ptr(stream))
    return H.reshape(phi.shape[:-2])


def lattice_torque(phi: torch.Tensor, g: torch.Tensor, q: float = 0.5, J: float = 1.0,
                   stream=None) -> torch.Tensor:
    """g_k * dH_k/dphi for a [..., Ly, Lx] float32 CUDA tensor (g: FP64 weights per grid)."""
    Ly, Lx = phi.shape[-2:]
    n = int(np.prod(phi.shape[:-2])) if phi.dim() > 2 else 1
    p = phi.contiguous()
    gg = g.reshape(-1).to(torch.float64).contiguous()
    grad = torch.empty_like(p)
    call("mpr_lattice_torque", n, int_array([Lx] * n), int_array([Ly] * n), _ptr(p), float(q),
         float(J), _ptr(gg), _ptr(grad), _stream_ptr(stream))
    return grad


def lattice_grad(phi: torch.Tensor, g: torch.Tensor, q: float = 0.5, J: float = 1.0,
                 want_phi: bool = True, want_J: bool = True, stream=None):
    """Both gradients of L = sum_k g_k H_k for a [..., Ly, Lx] float32 CUDA tensor:
    (dL/dphi or None, dL/dJ as a float64 [1] device tensor or None), from one kernel."""
    Ly, Lx = phi.shape[-2:]
    n = int(np.prod(phi.shape[:-2])) if phi.dim() > 2 else 1
    p = phi.contiguous()
    gg = g.reshape(-1).to(torch.float64).contiguous()
    gp = torch.empty_like(p) if want_phi else None
    gJ = torch.empty(1, dtype=torch.float64, device=phi.device) if want_J else None
    call("mpr_lattice_grad", n, int_array([Lx] * n), int_array([Ly] * n), _ptr(p), float(q),
         float(J), _ptr(gg), _ptr(gp) if gp is not None else None,
         _ptr(gJ) if gJ is not None else None, _stream_ptr(stream))
    return gp, gJ


class MPREnergy(torch.autograd.Function):
    """H(phi, J) = -J sum_<ij> cos(q (phi_i - phi_j)) with a hand-written backward.

    forward returns H per grid (FP64); backward returns, from the library's
    gradient kernel, the torque dH/dphi_i = J q sum_j sin(q (phi_i - phi_j))
    and dH/dJ = -sum_<ij> cos(q (phi_i - phi_j)), each weighted by the
    upstream gradient.
    """

    @staticmethod
    def forward(ctx, phi, J, q=0.5):
        Jv = float(J.item()) if isinstance(J, torch.Tensor) else float(J)
        H = lattice_energy(phi, q=q, J=Jv)
        ctx.save_for_backward(phi)
        ctx.q = q
        ctx.J = Jv
        ctx.J_tensor = J if isinstance(J, torch.Tensor) else None
        return H

    @staticmethod
    def backward(ctx, gH):
        (phi,) = ctx.saved_tensors
        want_J = ctx.J_tensor is not None and ctx.needs_input_grad[1]
        g_phi, g_J = lattice_grad(phi, gH.to(torch.float64), q=ctx.q, J=ctx.J,
                                  want_phi=ctx.needs_input_grad[0], want_J=want_J)
        if g_J is not None:
            J = ctx.J_tensor
            g_J = g_J.reshape(J.shape).to(device=J.device, dtype=J.dtype)
        return g_phi, g_J, None


def math_probe(fn: int, a: torch.Tensor, b: torch.Tensor = None) -> torch.Tensor:
    """The library's own approximations (fn 0: atan2, 2: series sine) or CUDA's (1, 3)."""
    a = a.to(torch.float32).contiguous()
    bb = b.to(torch.float32).contiguous() if b is not None else None
    out = torch.empty_like(a)
    call("mpr_math_probe", int(fn), a.numel(), _ptr(a), _ptr(bb) if bb is not None else None,
         _ptr(out), _stream_ptr(None))
    return out


def sample_energy_noalloc(z, gap, q: float = 0.5, J: float = 1.0, out=None, shapes=None,
                          stream=None):
    """e_s, N_SP, z_min, z_max per image from the library's allocation-free entry point.

    z, gap: either one concatenated pair of 1-D CUDA tensors (float32 values,
    uint8 mask, images in order) with ``shapes`` = [(Ly, Lx), ...], or
    sequences of 2-D CUDA tensors.  With the concatenated form and a
    preallocated ``out`` (dict of device tensors e_s float64[n], n_sp
    int64[n], zmin float32[n], zmax float32[n]) neither the library nor this
    wrapper allocates anything; the sequence form concatenates the images
    first (a torch allocation, made on the stream the call runs on).
    """
    st = stream if stream is not None else torch.cuda.current_stream()
    if shapes is None:
        zs, gs = _as_list(z), _as_list(gap)
        shapes = [tuple(int(v) for v in g.shape) for g in gs]
        with torch.cuda.stream(st):
            zf = torch.cat([t.reshape(-1).to(torch.float32) for t in zs])
            gf = torch.cat([(t.reshape(-1) != 0).to(torch.uint8) for t in gs])
    else:
        zf, gf = z, gap
        if not (zf.is_contiguous() and gf.is_contiguous() and zf.dtype == torch.float32
                and gf.dtype == torch.uint8):
            raise ValueError("concatenated inputs must be contiguous float32 values and uint8 masks")
    n = len(shapes)
    if out is None:
        dev = zf.device
        with torch.cuda.stream(st):
            out = dict(e_s=torch.empty(n, dtype=torch.float64, device=dev),
                       n_sp=torch.empty(n, dtype=torch.int64, device=dev),
                       zmin=torch.empty(n, dtype=torch.float32, device=dev),
                       zmax=torch.empty(n, dtype=torch.float32, device=dev))
    call("mpr_sample_energy_noalloc", n, int_array([s[1] for s in shapes]),
         int_array([s[0] for s in shapes]), _ptr(zf), _ptr(gf), float(q), float(J),
         _ptr(out["e_s"]), _ptr(out["n_sp"]), _ptr(out["zmin"]), _ptr(out["zmax"]),
         _stream_ptr(st))
    # keep the inputs alive until the kernels that read them have run
    for t in (zf, gf):
        t.record_stream(st)
    return out


def philox(ctr: np.ndarray, key, reference: bool = False) -> np.ndarray:
    """Philox4x32-10 blocks computed on the GPU (reference=True: the CUDA toolkit's routine)."""
    c = torch.as_tensor(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32), device="cuda")
    out = torch.empty_like(c)
    k = (C.c_uint32 * 2)(int(key[0]), int(key[1]))
    n = c.numel() // 4
    call("mpr_philox", n, _ptr(c), k, _ptr(out), int(reference), _stream_ptr(None))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(-1, 4)
