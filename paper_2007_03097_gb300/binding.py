"""Thin ctypes binding of the C ABI in ``include/sph.h``.

Argument marshalling only: every step of the SPH path runs in the CUDA
library ``lib/libsph.so``.  PyTorch provides device memory and streams.  The
functions keep the C names (``sph_create``, ``sph_build_tree``, ...); the
``Particles`` class owns the structure-of-arrays tensors that the C struct
``sph_particles`` points into.  There is no CPU fallback: a missing library
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

SPH_OK, SPH_ERR_ARG, SPH_ERR_CUDA, SPH_ERR_CAPACITY = 0, -1, -2, -3
SPH_ERR_NOT_CONVERGED, SPH_ERR_H_BOUNDS, SPH_ERR_NONFINITE, SPH_ERR_STATE = -4, -5, -6, -7
SPH_FP64, SPH_MIXED = 0, 1
SPH_ENERGY_INTERNAL, SPH_ENERGY_TOTAL = 0, 1
SPH_CURVE_MORTON, SPH_CURVE_HILBERT = 0, 1
SPH_HNET_NPARAM = 4609
SPH_HNET_SEED, SPH_HNET_TRAIN = 1, 2

_c = ctypes
_lib = None


class SphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class sph_params(_c.Structure):
    _fields_ = [("kernel", _c.c_int32), ("precision", _c.c_int32), ("periodic", _c.c_int32),
                ("fixed_h", _c.c_int32), ("box_lo", _c.c_double * 3), ("box_hi", _c.c_double * 3),
                ("gamma", _c.c_double), ("eta", _c.c_double), ("alpha", _c.c_double), ("beta", _c.c_double),
                ("eps_visc", _c.c_double), ("cfl", _c.c_double), ("h_tol", _c.c_double),
                ("max_sweeps", _c.c_int32), ("leaf_size", _c.c_int32), ("h_min", _c.c_double),
                ("h_max", _c.c_double), ("skin", _c.c_double), ("rho_ref", _c.c_double),
                ("nb_capacity", _c.c_int64), ("hnet_lr", _c.c_double), ("hnet_batch", _c.c_int32),
                ("hnet_iters", _c.c_int32), ("energy", _c.c_int32), ("curve", _c.c_int32),
                ("dim", _c.c_int32), ("pad", _c.c_int32)]


_FIELDS = ["vx", "vy", "vz", "m", "h", "u", "hprev", "rho", "omega", "P", "c", "ax", "ay", "az", "dudt",
           "divv", "vsig"]


class sph_particles(_c.Structure):
    _fields_ = [("n", _c.c_int64), ("x", _c.c_void_p), ("y", _c.c_void_p), ("z", _c.c_void_p)] + \
               [(f, _c.c_void_p) for f in _FIELDS] + [("nnb", _c.c_void_p), ("id", _c.c_void_p)]


class sph_density_stats(_c.Structure):
    _fields_ = [("sweeps", _c.c_int32), ("list_builds", _c.c_int32), ("n_unconverged", _c.c_int64),
                ("n_hbounds", _c.c_int64), ("interactions", _c.c_int64), ("list_entries", _c.c_int64),
                ("evaluations", _c.c_int64), ("launches", _c.c_int64), ("ms", _c.c_double),
                ("kernel_ms", _c.c_double), ("lists_ms", _c.c_double)]


class sph_force_stats(_c.Structure):
    _fields_ = [("interactions", _c.c_int64), ("list_entries", _c.c_int64), ("launches", _c.c_int64),
                ("ms", _c.c_double), ("kernel_ms", _c.c_double)]


class sph_step_stats(_c.Structure):
    _fields_ = [("dt", _c.c_double), ("dt_next", _c.c_double), ("momentum", _c.c_double * 3),
                ("force", _c.c_double * 3), ("energy", _c.c_double), ("power", _c.c_double),
                ("hnet_used", _c.c_int32), ("hnet_fallback", _c.c_int32), ("hnet_loss", _c.c_float),
                ("tree_moved", _c.c_int32), ("launches", _c.c_int64), ("density", sph_density_stats),
                ("forces", sph_force_stats), ("ms_tree", _c.c_double), ("ms_hnet", _c.c_double),
                ("ms_total", _c.c_double)]


EXPORTED = ["sph_create", "sph_destroy", "sph_set_params", "sph_last_error", "sph_version", "sph_build_tree",
            "sph_density", "sph_forces", "sph_step", "sph_totals", "sph_morton_keys", "sph_sort_keys",
            "sph_tree_info", "sph_list_info", "sph_export_leaves", "sph_neighbors", "sph_hnet_set_weights",
            "sph_hnet_get_weights", "sph_hnet_features", "sph_hnet_infer", "sph_hnet_seed", "sph_hnet_grad",
            "sph_hnet_train_step", "sph_sort_keys_noalloc", "sph_peak_fp32", "sph_test_hooks"]
SPH_SORT_NOALLOC_MAX = 262144


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(this package has no CPU fallback)")
    lib = _c.CDLL(path)
    V, I64, I32 = _c.c_void_p, _c.c_int64, _c.c_int
    sig = {
        "sph_create": ([_c.POINTER(sph_params), I64, _c.POINTER(V)], I32),
        "sph_destroy": ([V], None),
        "sph_set_params": ([V, _c.POINTER(sph_params)], I32),
        "sph_last_error": ([V], _c.c_char_p),
        "sph_version": ([], _c.c_char_p),
        "sph_build_tree": ([V, _c.POINTER(sph_particles), V], I32),
        "sph_density": ([V, _c.POINTER(sph_particles), V, _c.POINTER(sph_density_stats), V], I32),
        "sph_forces": ([V, _c.POINTER(sph_particles), _c.POINTER(sph_force_stats), V], I32),
        "sph_step": ([V, _c.POINTER(sph_particles), _c.c_double, I32, _c.POINTER(sph_step_stats), V], I32),
        "sph_totals": ([V, _c.POINTER(sph_particles), _c.POINTER(_c.c_double), V], I32),
        "sph_morton_keys": ([V, _c.POINTER(sph_particles), V, _c.POINTER(_c.c_double), V], I32),
        "sph_sort_keys": ([V, I64, V, V, V, V], I32),
        "sph_tree_info": ([V, _c.POINTER(I64), _c.POINTER(I64)], I32),
        "sph_list_info": ([V, _c.POINTER(I64), _c.POINTER(I64), _c.POINTER(I64), _c.POINTER(I32), _c.POINTER(I32),
                           _c.POINTER(I32), _c.POINTER(I32)],
                          I32),
        "sph_export_leaves": ([V, V, V, V], I32),
        "sph_neighbors": ([V, _c.POINTER(sph_particles), I32, V, V, V, V], I32),
        "sph_hnet_set_weights": ([V, V, I64], I32),
        "sph_hnet_get_weights": ([V, V, I64], I32),
        "sph_hnet_features": ([V, _c.POINTER(sph_particles), _c.c_double, V, V], I32),
        "sph_hnet_infer": ([V, V, I64, V, V], I32),
        "sph_hnet_seed": ([V, _c.POINTER(sph_particles), _c.c_double, V, _c.POINTER(I64), V], I32),
        "sph_hnet_grad": ([V, V, V, I64, V, V, V], I32),
        "sph_hnet_train_step": ([V, V, V, I64, _c.c_float, V, V], I32),
        "sph_sort_keys_noalloc": ([I64, V, V, V, V], I32),
        "sph_peak_fp32": ([_c.POINTER(_c.c_double), _c.POINTER(_c.c_double), V], I32),
        "sph_test_hooks": ([V, I32], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _stream(stream, device=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def make_params(p: dict) -> sph_params:
    """sph_params from a workload parameter dict (defaults for missing keys)."""
    q = sph_params()
    q.kernel = int(p.get("kernel", 0))
    q.precision = SPH_MIXED if p.get("precision", "fp64") in ("mixed", SPH_MIXED) else SPH_FP64
    q.periodic = int(bool(p.get("periodic", True)))
    q.fixed_h = int(bool(p.get("fixed_h", False)))
    q.box_lo = (_c.c_double * 3)(*p.get("box_lo", (0.0, 0.0, 0.0)))
    q.box_hi = (_c.c_double * 3)(*p.get("box_hi", (1.0, 1.0, 1.0)))
    q.gamma = float(p.get("gamma", 5.0 / 3.0))
    q.eta = float(p.get("eta", 1.2))
    q.alpha = float(p.get("alpha", 1.0))
    q.beta = float(p.get("beta", 2.0))
    q.eps_visc = float(p.get("eps_visc", 0.01))
    q.cfl = float(p.get("cfl", 0.3))
    q.h_tol = float(p.get("h_tol", 1e-6))
    q.max_sweeps = int(p.get("max_sweeps", 30))
    q.leaf_size = int(p.get("leaf_size", 32))
    q.h_min = float(p.get("h_min", 1e-6))
    q.h_max = float(p.get("h_max", 0.25))
    q.skin = float(p.get("skin", 0.05))
    q.rho_ref = float(p.get("rho_ref", 1.0))
    q.nb_capacity = int(p.get("nb_capacity", 0))
    q.hnet_lr = float(p.get("hnet_lr", 1e-3))
    q.hnet_batch = int(p.get("hnet_batch", 32768))
    q.hnet_iters = int(p.get("hnet_iters", 1))
    q.energy = int(p.get("energy", SPH_ENERGY_INTERNAL))
    curve = p.get("curve", SPH_CURVE_MORTON)
    q.curve = int({"morton": SPH_CURVE_MORTON, "hilbert": SPH_CURVE_HILBERT}.get(curve, curve))
    q.dim = int(p.get("dim", 3))
    return q


def _check(ctx, status: int, allow=()):
    if status != SPH_OK and status not in allow:
        msg = load().sph_last_error(ctx.handle if isinstance(ctx, Context) else ctx)
        raise SphError(status, msg.decode() if msg else "")
    return status


class Context:
    """Owner of an ``sph_ctx`` (all scratch memory for up to n_max particles)."""

    def __init__(self, params: dict, n_max: int):
        lib = load()
        self.params = dict(params)
        self.cparams = make_params(params)
        self.fp64 = self.cparams.precision == SPH_FP64
        h = _c.c_void_p()
        st = lib.sph_create(_c.byref(self.cparams), int(n_max), _c.byref(h))
        if st != SPH_OK:
            raise SphError(st, "sph_create failed (check parameters and device memory)")
        self.handle = h
        self.n_max = int(n_max)

    def close(self):
        if getattr(self, "handle", None):
            load().sph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: dict):
        q = make_params(params)
        _check(self, load().sph_set_params(self.handle, _c.byref(q)))
        self.params, self.cparams = dict(params), q


class Particles:
    """Device SoA particle arrays (torch tensors) and the matching C struct.

    All arrays are views into one device slab (``self.slab``, bytes), each
    starting on a 256-byte boundary, so that the whole state moves between
    host and device in one copy each way."""

    ALIGN = 256

    def __init__(self, n: int, fp64: bool, device="cuda"):
        self.n = int(n)
        self.fp64 = fp64
        self.dtype = torch.float64 if fp64 else torch.float32
        dev = torch.device(device)
        layout = [(f, torch.float64) for f in ("x", "y", "z")] + [(f, self.dtype) for f in _FIELDS] + \
                 [("nnb", torch.int32), ("id", torch.int32)]
        offs, off = [], 0
        for _, dt in layout:
            offs.append(off)
            nbytes = self.n * torch.empty(0, dtype=dt).element_size()
            off += (nbytes + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        self.slab = torch.zeros(max(off, self.ALIGN), dtype=torch.uint8, device=dev)
        for (f, dt), o in zip(layout, offs):
            nbytes = self.n * torch.empty(0, dtype=dt).element_size()
            setattr(self, f, self.slab[o:o + nbytes].view(dt))
        self.id.copy_(torch.arange(n, dtype=torch.int32, device=dev))

    @classmethod
    def from_workload(cls, w, fp64: bool, device="cuda") -> "Particles":
        p = cls(w.n, fp64, device)
        for f in ("x", "y", "z"):
            getattr(p, f).copy_(torch.from_numpy(np.ascontiguousarray(getattr(w, f))))
        for f in ("vx", "vy", "vz", "m", "h", "u"):
            getattr(p, f).copy_(torch.from_numpy(np.ascontiguousarray(getattr(w, f))).to(p.dtype))
        p.hprev.copy_(p.h)
        return p

    def struct(self) -> sph_particles:
        s = sph_particles()
        s.n = self.n
        s.x, s.y, s.z = self.x.data_ptr(), self.y.data_ptr(), self.z.data_ptr()
        for f in _FIELDS:
            setattr(s, f, getattr(self, f).data_ptr())
        s.nnb = self.nnb.data_ptr()
        s.id = self.id.data_ptr()
        return s

    def numpy(self, fields=None) -> dict:
        fields = fields or ["x", "y", "z"] + _FIELDS + ["nnb", "id"]
        out = {}
        for f in fields:
            t = getattr(self, f)
            a = t.cpu().numpy()
            out[f] = a.view(np.uint32) if f == "id" else (a.astype(np.float64) if a.dtype == np.float32 else a)
        return out

    def in_original_order(self, fields=None) -> dict:
        d = self.numpy(fields)
        order = np.argsort(self.id.cpu().numpy().view(np.uint32), kind="stable")
        return {k: v[order] for k, v in d.items()}


# ---------------------------------------------------------------------------- C names
def sph_version() -> str:
    return load().sph_version().decode()


def sph_create(params: dict, n_max: int) -> Context:
    return Context(params, n_max)


def sph_destroy(ctx: Context):
    ctx.close()


def _match(ctx: Context, p: Particles):
    if p.fp64 != ctx.fp64:
        raise ValueError("particle arrays are %s but the context computes in %s"
                         % ("FP64" if p.fp64 else "FP32", "SPH_FP64" if ctx.fp64 else "SPH_MIXED"))


def sph_build_tree(ctx: Context, p: Particles, stream=None):
    _match(ctx, p)
    s = p.struct()
    _check(ctx, load().sph_build_tree(ctx.handle, _c.byref(s), _stream(stream)))


def sph_density(ctx: Context, p: Particles, h_seed: torch.Tensor | None = None, stream=None,
                allow=(SPH_ERR_H_BOUNDS,)) -> dict:
    _match(ctx, p)
    s = p.struct()
    st = sph_density_stats()
    seed = h_seed.data_ptr() if h_seed is not None else None
    code = _check(ctx, load().sph_density(ctx.handle, _c.byref(s), seed, _c.byref(st), _stream(stream)), allow)
    return _as_dict(st) | {"status": code}


def sph_forces(ctx: Context, p: Particles, stream=None) -> dict:
    _match(ctx, p)
    s = p.struct()
    st = sph_force_stats()
    _check(ctx, load().sph_forces(ctx.handle, _c.byref(s), _c.byref(st), _stream(stream)))
    return _as_dict(st)


def sph_step(ctx: Context, p: Particles, dt: float, use_hnet: int = 0, stream=None,
             allow=(SPH_ERR_H_BOUNDS,)) -> dict:
    """use_hnet: bit set of SPH_HNET_SEED (seed h from the network) and
    SPH_HNET_TRAIN (one online training round after the step)."""
    _match(ctx, p)
    s = p.struct()
    st = sph_step_stats()
    code = _check(ctx, load().sph_step(ctx.handle, _c.byref(s), float(dt), int(use_hnet), _c.byref(st),
                                       _stream(stream)), allow)
    return _as_dict(st) | {"status": code}


def sph_totals(ctx: Context, p: Particles, stream=None) -> np.ndarray:
    s = p.struct()
    out = (_c.c_double * 8)()
    _check(ctx, load().sph_totals(ctx.handle, _c.byref(s), out, _stream(stream)))
    return np.array(out[:])


def sph_morton_keys(ctx: Context, p: Particles, stream=None):
    s = p.struct()
    keys = torch.empty(p.n, dtype=torch.int64, device=p.x.device)
    dom = (_c.c_double * 4)()
    _check(ctx, load().sph_morton_keys(ctx.handle, _c.byref(s), keys.data_ptr(), dom, _stream(stream)))
    torch.cuda.synchronize()
    return keys.cpu().numpy().view(np.uint64), np.array(dom[:])


def sph_sort_keys(ctx: Context, keys: torch.Tensor, ids: torch.Tensor | None, stream=None) -> torch.Tensor:
    n = keys.numel()
    perm = torch.empty(n, dtype=torch.int32, device=keys.device)
    _check(ctx, load().sph_sort_keys(ctx.handle, n, keys.data_ptr(), ids.data_ptr() if ids is not None else None,
                                     perm.data_ptr(), _stream(stream)))
    return perm


def sph_sort_keys_noalloc(keys: torch.Tensor, ids: torch.Tensor | None, stream=None,
                          perm: torch.Tensor | None = None) -> torch.Tensor:
    """(key, id) sort permutation without a context or any device allocation
    by the library (the permutation tensor here is the caller's own; pass
    ``perm`` to reuse one).  Runs on the keys' device, on ``stream`` or that
    device's current stream."""
    n = keys.numel()
    with torch.cuda.device(keys.device):
        if perm is None:
            perm = torch.empty(n, dtype=torch.int32, device=keys.device)
        st = load().sph_sort_keys_noalloc(n, keys.data_ptr(), ids.data_ptr() if ids is not None else None,
                                           perm.data_ptr(), _stream(stream, keys.device))
        if st != SPH_OK:
            raise SphError(st, load().sph_last_error(None).decode())
    return perm


SPH_TEST_SKIP_MMA = 1


def sph_test_hooks(ctx: Context, flags: int) -> None:
    _check(ctx, load().sph_test_hooks(ctx.handle, int(flags)))


def sph_peak_fp32(stream=None) -> dict:
    """Measured FP32 fused multiply-add rate of the current device (TFLOP/s)."""
    tf, ms = _c.c_double(), _c.c_double()
    st = load().sph_peak_fp32(_c.byref(tf), _c.byref(ms), _stream(stream))
    if st != SPH_OK:
        raise SphError(st, "sph_peak_fp32 failed")
    return {"tflops": float(tf.value), "ms": float(ms.value)}


def sph_tree_info(ctx: Context):
    nl, ng = _c.c_int64(), _c.c_int64()
    _check(ctx, load().sph_tree_info(ctx.handle, _c.byref(nl), _c.byref(ng)))
    return int(nl.value), int(ng.value)


def sph_list_info(ctx: Context) -> dict:
    """Neighbour-list slots reserved and used by the last build, whether the
    context sizes lists by exact counts, and whether the last build predicted
    its widths from the neighbour counts (with the predicted builds that
    overflowed)."""
    r, u, un = _c.c_int64(), _c.c_int64(), _c.c_int64()
    e, um, pr, pf = _c.c_int32(), _c.c_int32(), _c.c_int32(), _c.c_int32()
    _check(ctx, load().sph_list_info(ctx.handle, _c.byref(r), _c.byref(u), _c.byref(un), _c.byref(e),
                                     _c.byref(um), _c.byref(pr), _c.byref(pf)))
    return {"slots_reserved": int(r.value), "slots_used": int(u.value), "union_used": int(un.value),
            "exact_sizing": bool(e.value), "union_max": int(um.value), "predicted": bool(pr.value),
            "pred_failures": int(pf.value)}


def sph_export_leaves(ctx: Context, stream=None):
    nl, _ = sph_tree_info(ctx)
    lb = torch.empty(nl + 1, dtype=torch.int32, device="cuda")
    lv = torch.empty(max(nl, 1), dtype=torch.int32, device="cuda")
    _check(ctx, load().sph_export_leaves(ctx.handle, lb.data_ptr(), lv.data_ptr(), _stream(stream)))
    return lb.cpu().numpy(), lv[:nl].cpu().numpy()


def sph_neighbors(ctx: Context, p: Particles, kind: int, stream=None):
    """Exact neighbour sets as CSR (counts, offsets, idx) in the current order."""
    s = p.struct()
    lib = load()
    counts = torch.zeros(p.n, dtype=torch.int64, device=p.x.device)
    _check(ctx, lib.sph_neighbors(ctx.handle, _c.byref(s), int(kind), counts.data_ptr(), None, None,
                                  _stream(stream)))
    offsets = torch.zeros(p.n + 1, dtype=torch.int64, device=p.x.device)
    offsets[1:] = torch.cumsum(counts, 0)
    total = int(offsets[-1].item())
    idx = torch.empty(max(total, 1), dtype=torch.int32, device=p.x.device)
    _check(ctx, lib.sph_neighbors(ctx.handle, _c.byref(s), int(kind), counts.data_ptr(), offsets.data_ptr(),
                                  idx.data_ptr(), _stream(stream)))
    torch.cuda.synchronize()
    return counts.cpu().numpy(), offsets.cpu().numpy(), idx[:total].cpu().numpy()


def sph_hnet_set_weights(ctx: Context, theta) -> None:
    a = np.ascontiguousarray(theta, dtype=np.float32)
    _check(ctx, load().sph_hnet_set_weights(ctx.handle, a.ctypes.data, a.size))


def sph_hnet_get_weights(ctx: Context) -> np.ndarray:
    a = np.empty(SPH_HNET_NPARAM, dtype=np.float32)
    _check(ctx, load().sph_hnet_get_weights(ctx.handle, a.ctypes.data, a.size))
    return a


def sph_hnet_features(ctx: Context, p: Particles, dt: float, stream=None) -> torch.Tensor:
    s = p.struct()
    f = torch.empty((p.n, 5), dtype=torch.float32, device=p.x.device)
    _check(ctx, load().sph_hnet_features(ctx.handle, _c.byref(s), float(dt), f.data_ptr(), _stream(stream)))
    return f


def sph_hnet_infer(ctx: Context, feats: torch.Tensor, stream=None) -> torch.Tensor:
    feats = feats.contiguous()
    y = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
    _check(ctx, load().sph_hnet_infer(ctx.handle, feats.data_ptr(), feats.shape[0], y.data_ptr(), _stream(stream)))
    return y


def sph_hnet_seed(ctx: Context, p: Particles, dt: float, stream=None):
    """The h seed sph_step takes with SPH_HNET_SEED (device tensor of the
    particles' float type) and the number of particles that kept h."""
    _match(ctx, p)
    s = p.struct()
    seed = torch.empty(p.n, dtype=p.dtype, device=p.x.device)
    fb = _c.c_int64()
    _check(ctx, load().sph_hnet_seed(ctx.handle, _c.byref(s), float(dt), seed.data_ptr(), _c.byref(fb),
                                     _stream(stream)))
    return seed, int(fb.value)


def sph_hnet_grad(ctx: Context, feats: torch.Tensor, target: torch.Tensor, stream=None):
    feats, target = feats.contiguous(), target.contiguous()
    g = np.empty(SPH_HNET_NPARAM, dtype=np.float32)
    loss = _c.c_float()
    _check(ctx, load().sph_hnet_grad(ctx.handle, feats.data_ptr(), target.data_ptr(), feats.shape[0],
                                     g.ctypes.data, _c.byref(loss), _stream(stream)))
    return float(loss.value), g


def sph_hnet_train_step(ctx: Context, feats: torch.Tensor, target: torch.Tensor, lr: float, stream=None) -> float:
    feats, target = feats.contiguous(), target.contiguous()
    loss = _c.c_float()
    _check(ctx, load().sph_hnet_train_step(ctx.handle, feats.data_ptr(), target.data_ptr(), feats.shape[0],
                                           float(lr), _c.byref(loss), _stream(stream)))
    return float(loss.value)


def _as_dict(st) -> dict:
    out = {}
    for name, _ in st._fields_:
        v = getattr(st, name)
        if isinstance(v, _c.Structure):
            v = _as_dict(v)
        elif isinstance(v, _c.Array):
            v = list(v)
        out[name] = v
    return out
