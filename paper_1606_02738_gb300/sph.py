"""Thin ctypes binding of libsph (include/sph.h): same names, argument
marshalling only. Every step of the computation runs in the CUDA library;
there is no CPU fallback -- if the library cannot be loaded, calls raise.

Device buffers are torch CUDA tensors (the binding passes their data
pointers); the stream is torch's current CUDA stream unless one is given.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

SPH_OK = 0
SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_ENOTCONVERGED = -1, -2, -3, -4
SPH_EBOXTOOSMALL, SPH_ENONPHYSICAL, SPH_ETIMEOUT, SPH_ESTATE = -5, -6, -7, -8
ERROR_NAMES = {SPH_EINVAL: "SPH_EINVAL", SPH_ENOMEM: "SPH_ENOMEM", SPH_ECUDA: "SPH_ECUDA",
               SPH_ENOTCONVERGED: "SPH_ENOTCONVERGED", SPH_EBOXTOOSMALL: "SPH_EBOXTOOSMALL",
               SPH_ENONPHYSICAL: "SPH_ENONPHYSICAL", SPH_ETIMEOUT: "SPH_ETIMEOUT",
               SPH_ESTATE: "SPH_ESTATE"}

SPH_X, SPH_V, SPH_U, SPH_H, SPH_RHO, SPH_OMEGA, SPH_P, SPH_A, SPH_DUDT = range(9)
SPH_NNGB, SPH_NITER, SPH_NFORCE, SPH_M, SPH_CELL, SPH_LEAF_CELL = 9, 10, 11, 12, 13, 14
SPH_MODE_PLAIN, SPH_MODE_BATCHED, SPH_MODE_SYMMETRIC = 0, 1, 2
SPH_PREC_FP32, SPH_PREC_KAHAN = 0, 1

# field -> (dtype name, components)
FIELDS = {SPH_X: ("float64", 3), SPH_V: ("float32", 3), SPH_U: ("float32", 1),
          SPH_H: ("float64", 1), SPH_RHO: ("float32", 1), SPH_OMEGA: ("float32", 1),
          SPH_P: ("float32", 1), SPH_A: ("float32", 3), SPH_DUDT: ("float32", 1),
          SPH_NNGB: ("int32", 1), SPH_NITER: ("int32", 1), SPH_NFORCE: ("int32", 1),
          SPH_M: ("float32", 1), SPH_CELL: ("int32", 4), SPH_LEAF_CELL: ("int32", 3)}
FIELD_NAMES = {"x": SPH_X, "v": SPH_V, "u": SPH_U, "h": SPH_H, "rho": SPH_RHO,
               "omega": SPH_OMEGA, "P": SPH_P, "a": SPH_A, "dudt": SPH_DUDT,
               "nngb": SPH_NNGB, "niter": SPH_NITER, "nforce": SPH_NFORCE, "m": SPH_M,
               "cell": SPH_CELL, "leaf_cell": SPH_LEAF_CELL}


class sph_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("n_ngb", ctypes.c_double),
                ("h_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("n_split", ctypes.c_int), ("precision", ctypes.c_int),
                ("mode", ctypes.c_int), ("profile", ctypes.c_int),
                ("pair_sort", ctypes.c_int), ("reuse_grid", ctypes.c_int),
                ("tile", ctypes.c_int), ("cell_factor", ctypes.c_double),
                ("reuse_lists", ctypes.c_int), ("work_queue", ctypes.c_int)]


class sph_stats_t(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_boxes", ctypes.c_int64),
                ("n_top_cells", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_pairs_density", ctypes.c_int64), ("n_pairs_force", ctypes.c_int64),
                ("density_interactions", ctypes.c_int64), ("force_interactions", ctypes.c_int64),
                ("density_pair_candidates", ctypes.c_int64),
                ("force_pair_candidates", ctypes.c_int64),
                ("density_passes", ctypes.c_int32), ("rebuilds", ctypes.c_int32),
                ("max_iter_used", ctypes.c_int32), ("batched_fallbacks", ctypes.c_int32),
                ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
                ("stage_max_density", ctypes.c_int32), ("stage_max_force", ctypes.c_int32),
                ("total_density_interactions", ctypes.c_int64),
                ("total_force_interactions", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("density_launches", ctypes.c_int64),
                ("force_launches", ctypes.c_int64),
                ("t_grid_ms", ctypes.c_double), ("t_lists_ms", ctypes.c_double),
                ("t_density_ms", ctypes.c_double), ("t_ghost_ms", ctypes.c_double),
                ("t_force_ms", ctypes.c_double), ("t_integrate_ms", ctypes.c_double),
                ("t_sort_ms", ctypes.c_double),
                ("direct_list_warps", ctypes.c_int32), ("direct_stage_warps", ctypes.c_int32),
                ("fallback_causes", ctypes.c_int32 * 4),
                ("tier2_groups", ctypes.c_int32 * 2), ("tier3_entries", ctypes.c_int32 * 2),
                ("sort_launches", ctypes.c_int64), ("reused_steps", ctypes.c_int64),
                ("redone_steps", ctypes.c_int64), ("graph_steps", ctypes.c_int64),
                ("n_groups", ctypes.c_int64), ("cache_density_groups", ctypes.c_int64),
                ("cache_force_groups", ctypes.c_int64), ("cache_built_groups", ctypes.c_int64),
                ("cache_relist_warps", ctypes.c_int64)]


class SphError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def header_functions() -> list[str]:
    """Names of the functions declared in include/sph.h."""
    hdr = os.path.join(_build.ROOT, "include", "sph.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", text)))


def lib(build_if_needed: bool = True):
    """Load libsph.so (building it first if sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsph not built ({path}); call paper_1606_02738_gb300.build.build()")
        L = ctypes.CDLL(path)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.sph_default_params.argtypes = [ctypes.POINTER(sph_params)]
        L.sph_default_params.restype = None
        L.sph_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(sph_params), P]
        L.sph_workspace_size.argtypes = [P, I64, I, ctypes.POINTER(ctypes.c_size_t)]
        L.sph_set_workspace.argtypes = [P, P, ctypes.c_size_t]
        L.sph_init.argtypes = [P, I, P, P, P, P, P, P, P]
        L.sph_density.argtypes = [P]
        L.sph_force.argtypes = [P]
        L.sph_step.argtypes = [P, D, I]
        L.sph_get.argtypes = [P, I, P]
        L.sph_get_pair_order.argtypes = [P, I, P, P]
        L.sph_autotune.argtypes = [P, P, P, P, P]
        L.sph_fp32_peak.argtypes = [I, P, P]
        L.sph_stats.argtypes = [P, ctypes.POINTER(sph_stats_t)]
        L.sph_grid.argtypes = [P, I, P, P]
        L.sph_last_error.argtypes = [P]
        L.sph_last_error.restype = ctypes.c_char_p
        L.sph_destroy.argtypes = [P]
        L.sph_destroy.restype = None
        for f in ("sph_create", "sph_workspace_size", "sph_set_workspace", "sph_init",
                  "sph_density", "sph_force", "sph_step", "sph_get", "sph_get_pair_order",
                  "sph_autotune", "sph_fp32_peak", "sph_stats", "sph_grid"):
            getattr(L, f).restype = I
        _lib = L
        return L


def _check(ctx, rc: int, where: str):
    if rc != SPH_OK:
        msg = lib().sph_last_error(ctx).decode() if ctx else ""
        raise SphError(rc, where, msg)


def _ptr(t) -> int:
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------- C ABI names

def sph_default_params() -> sph_params:
    p = sph_params()
    lib().sph_default_params(ctypes.byref(p))
    return p


def sph_create(params: sph_params | None = None, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    rc = lib().sph_create(ctypes.byref(ctx), ctypes.byref(params) if params else None,
                          _stream(stream))
    _check(None, rc, "sph_create")
    return ctx


def sph_workspace_size(ctx, n_total: int, n_boxes: int) -> int:
    b = ctypes.c_size_t()
    _check(ctx, lib().sph_workspace_size(ctx, n_total, n_boxes, ctypes.byref(b)),
           "sph_workspace_size")
    return int(b.value)


def sph_set_workspace(ctx, buf) -> None:
    _check(ctx, lib().sph_set_workspace(ctx, ctypes.c_void_p(_ptr(buf)), buf.numel() *
                                        buf.element_size()), "sph_set_workspace")


def sph_init(ctx, box_offsets, box_len, x, v, m, u, h) -> None:
    """box_offsets (n_boxes+1) and box_len (n_boxes, 3) are host arrays;
    x (N,3) float64, v (N,3) float32, m, u (N) float32, h (N) float64 are CUDA
    tensors in caller order."""
    offs = np.ascontiguousarray(box_offsets, dtype=np.int64)
    bl = np.ascontiguousarray(box_len, dtype=np.float64).reshape(-1, 3)
    nb = bl.shape[0]
    if offs.shape[0] != nb + 1:
        raise ValueError("box_offsets needs n_boxes + 1 entries")
    for t, dt in ((x, "float64"), (v, "float32"), (m, "float32"), (u, "float32"),
                  (h, "float64")):
        if not t.is_cuda or str(t.dtype) != f"torch.{dt}" or not t.is_contiguous():
            raise TypeError(f"expected a contiguous CUDA {dt} tensor, got {t.dtype} on {t.device}")
    rc = lib().sph_init(ctx, nb, offs.ctypes.data_as(ctypes.c_void_p),
                        bl.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(_ptr(x)),
                        ctypes.c_void_p(_ptr(v)), ctypes.c_void_p(_ptr(m)),
                        ctypes.c_void_p(_ptr(u)), ctypes.c_void_p(_ptr(h)))
    _check(ctx, rc, "sph_init")


def sph_density(ctx) -> None:
    _check(ctx, lib().sph_density(ctx), "sph_density")


def sph_force(ctx) -> None:
    _check(ctx, lib().sph_force(ctx), "sph_force")


def sph_step(ctx, dt: float, n_steps: int = 1) -> None:
    _check(ctx, lib().sph_step(ctx, float(dt), int(n_steps)), "sph_step")


def sph_get(ctx, field: int, out) -> None:
    _check(ctx, lib().sph_get(ctx, int(field), ctypes.c_void_p(_ptr(out))), "sph_get")


def sph_get_pair_order(ctx, axis: int, order_out, leaf_out) -> None:
    """order_out, leaf_out: int32 CUDA tensors of N entries (store slot order)."""
    for t in (order_out, leaf_out):
        if not t.is_cuda or str(t.dtype) != "torch.int32" or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA int32 tensors")
    _check(ctx, lib().sph_get_pair_order(ctx, int(axis), ctypes.c_void_p(_ptr(order_out)),
                                         ctypes.c_void_p(_ptr(leaf_out))),
           "sph_get_pair_order")


def sph_autotune(ctx) -> dict:
    """Runs the library's autotuner on the loaded state; returns its choice."""
    tile, ns = ctypes.c_int(), ctypes.c_int()
    cf, ms = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().sph_autotune(ctx, ctypes.byref(tile), ctypes.byref(ns), ctypes.byref(cf),
                                   ctypes.byref(ms)), "sph_autotune")
    return {"tile": tile.value, "n_split": ns.value, "cell_factor": cf.value,
            "best_ms": ms.value}


def sph_fp32_peak(device: int = 0) -> dict:
    """Measured FP32 FFMA rate of a device (TFLOP/s) and the best launch time."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(None, lib().sph_fp32_peak(int(device), ctypes.byref(tf), ctypes.byref(ms)),
           "sph_fp32_peak")
    return {"tflops": tf.value, "ms": ms.value}


def sph_stats(ctx) -> dict:
    s = sph_stats_t()
    _check(ctx, lib().sph_stats(ctx, ctypes.byref(s)), "sph_stats")
    out = {}
    for name, _ in sph_stats_t._fields_:
        v = getattr(s, name)
        out[name] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def sph_grid(ctx, box: int = 0) -> dict:
    """Top grid of one box as of the last regrid: cells per axis and FP64 widths."""
    n = (ctypes.c_int32 * 3)()
    w = (ctypes.c_double * 3)()
    _check(ctx, lib().sph_grid(ctx, int(box), n, w), "sph_grid")
    return {"n": list(n), "w": list(w)}


def sph_last_error(ctx) -> str:
    return lib().sph_last_error(ctx).decode()


def sph_destroy(ctx) -> None:
    if ctx:
        lib().sph_destroy(ctx)


SPH_NOALLOC_MAX_PARTICLES = 16384


def sph_density_noalloc(box_len, x, m, h0, h_out, rho_out, omega_out, n_ngb: float = 48.0,
                        h_tol: float = 1e-6, max_iter: int = 30, stream=None) -> None:
    """Allocation-free density stage for one small box (see include/sph.h):
    x (N,3) float64, m (N) float32, h0 (N) float64 in; h_out (N) float64,
    rho_out, omega_out (N) float32 out -- all CUDA tensors the caller owns."""
    L = lib()
    f = L.sph_density_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    box = np.ascontiguousarray(box_len, dtype=np.float64).reshape(3)
    rc = f(int(x.shape[0]), box.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(_ptr(x)),
           ctypes.c_void_p(_ptr(m)), ctypes.c_void_p(_ptr(h0)), float(n_ngb), float(h_tol),
           int(max_iter), ctypes.c_void_p(_ptr(h_out)), ctypes.c_void_p(_ptr(rho_out)),
           ctypes.c_void_p(_ptr(omega_out)), _stream(stream))
    if rc != SPH_OK:
        raise SphError(rc, "sph_density_noalloc", "")


# ------------------------------------------------- convenience (marshalling)

class Context:
    """Owns one sph_ctx; moves a particle set onto the device and reads
    fields back as torch tensors in caller order."""

    def __init__(self, n_split: int = 64, precision: int = SPH_PREC_FP32,
                 mode: int = SPH_MODE_BATCHED, n_ngb: float = 48.0, gamma: float = 5.0 / 3.0,
                 h_tol: float = 1e-6, max_iter: int = 30, profile: bool = False,
                 pair_sort: bool = True, reuse_grid: bool = True, tile: int = 0,
                 cell_factor: float = 2.0, reuse_lists: int = 1, work_queue: int = 1,
                 stream=None, device="cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        p = sph_default_params()
        p.n_split, p.precision, p.mode = n_split, precision, mode
        p.profile = int(bool(profile))
        p.pair_sort = int(bool(pair_sort))
        p.reuse_grid = int(bool(reuse_grid))
        p.tile, p.cell_factor = int(tile), float(cell_factor)
        p.reuse_lists = int(reuse_lists)
        p.work_queue = int(work_queue)
        p.n_ngb, p.gamma, p.h_tol, p.max_iter = n_ngb, gamma, h_tol, max_iter
        self.params = p
        self.stream = stream
        self.ctx = sph_create(p, stream)
        self.n = 0

    def close(self):
        if self.ctx:
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, p):
        """Copy a generated ParticleSet to the device and call sph_init."""
        t = self.torch
        dev = self.device
        self._in = dict(
            x=t.as_tensor(p.x, dtype=t.float64).to(dev).contiguous(),
            v=t.as_tensor(p.v, dtype=t.float32).to(dev).contiguous(),
            m=t.as_tensor(p.m, dtype=t.float32).to(dev).contiguous(),
            u=t.as_tensor(p.u, dtype=t.float32).to(dev).contiguous(),
            h=t.as_tensor(p.h, dtype=t.float64).to(dev).contiguous())
        self.n = p.n
        sph_init(self.ctx, p.box_offsets, p.box, **self._in)
        return self

    def density(self):
        sph_density(self.ctx)

    def force(self):
        sph_force(self.ctx)

    def step(self, dt: float, n_steps: int = 1):
        sph_step(self.ctx, dt, n_steps)

    def get(self, name: str):
        f = FIELD_NAMES[name]
        dtype, comp = FIELDS[f]
        shape = (self.n, comp) if comp > 1 else (self.n,)
        out = self.torch.empty(shape, dtype=getattr(self.torch, dtype), device=self.device)
        sph_get(self.ctx, f, out)
        return out

    def autotune(self) -> dict:
        return sph_autotune(self.ctx)

    def pair_order(self, axis: int):
        """(order, leaf) int32 tensors of the pair-axis sort along `axis`."""
        order = self.torch.empty(self.n, dtype=self.torch.int32, device=self.device)
        leaf = self.torch.empty(self.n, dtype=self.torch.int32, device=self.device)
        sph_get_pair_order(self.ctx, axis, order, leaf)
        return order, leaf

    def stats(self) -> dict:
        return sph_stats(self.ctx)

    def grid(self, box: int = 0) -> dict:
        return sph_grid(self.ctx, box)
