"""Plain FP64 CPU oracle of the SPH hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. The CUDA library never calls it, and it
never calls the CUDA library: the two share no code, header or helper.

The arithmetic lives in `sph_oracle.c` (double precision, OpenMP over
particles); this module compiles it with gcc, loads it with ctypes, loops over
independent boxes and adds the kick-drift-kick update in NumPy float64.

Paper: Schaller, Gonnet, Chalk, Draper, "SWIFT: Using task-based parallelism,
fully asynchronous communication, and graph partition-based domain
decomposition for strong scaling on more than 100,000 cores", PASC '16.
  Section 2, Eq. (rho)            density sum             -> density()
  Section 2 (constant neighbours) smoothing-length root   -> density()
  Section 2, P_i and Omega_i      pressure, grad-h term   -> density(), force()
  Section 2, Eqs. (dvdt), (dudt)  accelerations, du/dt    -> force()
  Section 3.1, integrator task    kick/drift update       -> kdk_step()

Where the paper is silent this oracle reads it as follows: the smoothing
kernel is the cubic spline with support h; h solves (32/3) sum_j w(r_ij/h) =
n_ngb (48 by default), the weighted neighbour number, which is monotone in h
so the root is unique; the sums include j = i; the integrator is
kick-drift-kick with one global dt, and the mid-step force uses v and u
predicted to the end of the step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsph_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EBOXTOOSMALL, ENONPHYSICAL, ENOMEM = 0, -1, -2, -3, -4
_ERRORS = {EINVAL: "invalid argument", EBOXTOOSMALL: "smoothing length exceeds L/3",
           ENONPHYSICAL: "non-physical density or Omega", ENOMEM: "out of memory"}

H_TOL = 1e-13


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {_ERRORS.get(code, code)} ({code})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile sph_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        Ci = ctypes.c_int
        lib.or_version.restype = Ci
        lib.or_num_threads.restype = Ci
        lib.or_w_hat.argtypes = [I64, P, P, P]
        for f in (lib.or_W, lib.or_dWdr, lib.or_dWdh):
            f.argtypes = [D, D]
            f.restype = D
        lib.or_neighbours.argtypes = [I64, P, P, P, Ci, P, P, P]
        lib.or_neighbours.restype = Ci
        lib.or_density_fixed_h.argtypes = [I64, P, P, P, P, Ci, P, P, P, P, P]
        lib.or_density_fixed_h.restype = Ci
        lib.or_density.argtypes = [I64, P, P, P, D, D, Ci, P, P, P, P, P, P, P, P, I64]
        lib.or_density.restype = Ci
        lib.or_force.argtypes = [I64, P, P, P, P, P, P, P, P, D, Ci, P, P, P, P, I64]
        lib.or_force.restype = Ci
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().or_num_threads())


# ------------------------------------------------------------------ kernel

def w_hat(q) -> tuple[np.ndarray, np.ndarray]:
    """Dimensionless cubic spline w(q) and w'(q) (support q < 1)."""
    q = _f64(np.atleast_1d(q))
    w = np.empty_like(q)
    dw = np.empty_like(q)
    _load().or_w_hat(q.size, _p(q), _p(w), _p(dw))
    return w, dw


def W(r: float, h: float) -> float:
    """Smoothing kernel W(r, h) = (8/pi) w(r/h) / h^3."""
    return float(_load().or_W(float(r), float(h)))


def dWdr(r: float, h: float) -> float:
    return float(_load().or_dWdr(float(r), float(h)))


def dWdh(r: float, h: float) -> float:
    return float(_load().or_dWdh(float(r), float(h)))


# ------------------------------------------------------- single-box calls

def neighbours(x, L, R, use_tree: bool = True) -> list[np.ndarray]:
    """For every i, the sorted j != i with minimum-image r_ij < R[i]."""
    lib = _load()
    x = _f64(x)
    L = _f64(L)
    n = x.shape[0]
    R = _f64(np.broadcast_to(R, (n,)))
    counts = np.zeros(n, dtype=np.int64)
    rc = lib.or_neighbours(n, _p(x), _p(L), _p(R), int(use_tree), _p(counts), None, None)
    if rc:
        raise OracleError(rc, "neighbours")
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    idx = np.zeros(max(1, int(offs[-1])), dtype=np.int64)
    rc = lib.or_neighbours(n, _p(x), _p(L), _p(R), int(use_tree), _p(counts), _p(offs), _p(idx))
    if rc:
        raise OracleError(rc, "neighbours")
    return [np.sort(idx[offs[i]:offs[i + 1]]) for i in range(n)]


def density_fixed_h(x, m, L, h, use_tree: bool = True) -> dict:
    """Density sums at the given h (no root finding): rho, drho/dh, weighted
    neighbour number N(h), dN/dh and the neighbour count."""
    lib = _load()
    x, m, L, h = _f64(x), _f64(m), _f64(L), _f64(h)
    n = x.shape[0]
    out = {k: np.zeros(n) for k in ("rho", "drho_dh", "n_w", "dn_w_dh")}
    cnt = np.zeros(n, dtype=np.int64)
    rc = lib.or_density_fixed_h(n, _p(x), _p(m), _p(L), _p(h), int(use_tree), _p(out["rho"]),
                                _p(out["drho_dh"]), _p(out["n_w"]), _p(out["dn_w_dh"]), _p(cnt))
    if rc:
        raise OracleError(rc, "density_fixed_h")
    out["count"] = cnt
    return out


def density(x, m, L, h0, n_ngb: float = 48.0, tol: float = H_TOL, use_tree: bool = True,
            subset=None) -> dict:
    """Density stage: smoothing lengths with N_i(h_i) = n_ngb, then rho,
    drho/dh, Omega. `subset` (indices) limits the solve to those particles;
    the other entries of the outputs are NaN."""
    lib = _load()
    x, m, L = _f64(x), _f64(m), _f64(L)
    n = x.shape[0]
    h = _f64(np.broadcast_to(h0, (n,))).copy()
    fill = np.nan if subset is not None else 0.0
    out = {k: np.full(n, fill) for k in ("rho", "drho_dh", "omega", "n_w")}
    cnt = np.zeros(n, dtype=np.int64)
    it = np.zeros(n, dtype=np.int32)
    sub = None
    nsub = 0
    if subset is not None:
        sub = np.ascontiguousarray(subset, dtype=np.int64)
        nsub = sub.size
    rc = lib.or_density(n, _p(x), _p(m), _p(L), float(n_ngb), float(tol), int(use_tree), _p(h),
                        _p(out["rho"]), _p(out["drho_dh"]), _p(out["omega"]), _p(out["n_w"]),
                        _p(cnt), _p(it), _p(sub) if sub is not None else None, nsub)
    if rc:
        raise OracleError(rc, "density")
    if subset is not None:
        mask = np.ones(n, dtype=bool)
        mask[sub] = False
        h[mask] = np.nan
    out.update(h=h, count=cnt, iters=it)
    return out


def force(x, v, m, u, h, rho, omega, L, gamma: float, use_tree: bool = True,
          subset=None) -> dict:
    """Force stage (Eqs. dvdt, dudt): accelerations a (N,3), du/dt and the
    count of j != i with r_ij < max(h_i, h_j)."""
    lib = _load()
    x, v, m, u, h, rho, omega, L = map(_f64, (x, v, m, u, h, rho, omega, L))
    n = x.shape[0]
    fill = np.nan if subset is not None else 0.0
    a = np.full((n, 3), fill)
    dudt = np.full(n, fill)
    cnt = np.zeros(n, dtype=np.int64)
    sub = None
    nsub = 0
    if subset is not None:
        sub = np.ascontiguousarray(subset, dtype=np.int64)
        nsub = sub.size
    rc = lib.or_force(n, _p(x), _p(v), _p(m), _p(u), _p(h), _p(rho), _p(omega), _p(L),
                      float(gamma), int(use_tree), _p(a), _p(dudt), _p(cnt),
                      _p(sub) if sub is not None else None, nsub)
    if rc:
        raise OracleError(rc, "force")
    return {"a": a, "dudt": dudt, "count": cnt}


# ------------------------------------------------------------ whole sets

@dataclass
class State:
    """FP64 particle state of one or more independent periodic boxes."""
    x: np.ndarray
    v: np.ndarray
    m: np.ndarray
    u: np.ndarray
    h: np.ndarray
    box: np.ndarray
    box_offsets: np.ndarray
    gamma: float
    n_ngb: float
    rho: np.ndarray | None = None
    drho_dh: np.ndarray | None = None
    omega: np.ndarray | None = None
    a: np.ndarray | None = None
    dudt: np.ndarray | None = None
    n_dens: np.ndarray | None = None
    n_force: np.ndarray | None = None
    t: float = 0.0

    @classmethod
    def from_particles(cls, p) -> "State":
        """Upcast a generated particle set (float32 v, m, u) to float64."""
        return cls(x=_f64(p.x).copy(), v=_f64(p.v).copy(), m=_f64(p.m).copy(),
                   u=_f64(p.u).copy(), h=_f64(p.h).copy(), box=_f64(p.box).copy(),
                   box_offsets=np.asarray(p.box_offsets, dtype=np.int64).copy(),
                   gamma=float(p.gamma), n_ngb=float(p.n_ngb))

    def boxes(self):
        for b in range(self.box.shape[0]):
            yield b, slice(int(self.box_offsets[b]), int(self.box_offsets[b + 1]))


def compute_density(s: State, use_tree: bool = True) -> State:
    """h solve + rho, drho/dh, Omega for every box, in place."""
    n = s.x.shape[0]
    s.rho = np.zeros(n)
    s.drho_dh = np.zeros(n)
    s.omega = np.zeros(n)
    s.n_dens = np.zeros(n, dtype=np.int64)
    for b, sl in s.boxes():
        d = density(s.x[sl], s.m[sl], s.box[b], s.h[sl], s.n_ngb, use_tree=use_tree)
        s.h[sl] = d["h"]
        s.rho[sl] = d["rho"]
        s.drho_dh[sl] = d["drho_dh"]
        s.omega[sl] = d["omega"]
        s.n_dens[sl] = d["count"]
    return s


def compute_force(s: State, v=None, u=None, use_tree: bool = True) -> State:
    """a and du/dt for every box (velocities / energies default to the state's)."""
    v = s.v if v is None else v
    u = s.u if u is None else u
    n = s.x.shape[0]
    s.a = np.zeros((n, 3))
    s.dudt = np.zeros(n)
    s.n_force = np.zeros(n, dtype=np.int64)
    for b, sl in s.boxes():
        f = force(s.x[sl], v[sl], s.m[sl], u[sl], s.h[sl], s.rho[sl], s.omega[sl], s.box[b],
                  s.gamma, use_tree=use_tree)
        s.a[sl] = f["a"]
        s.dudt[sl] = f["dudt"]
        s.n_force[sl] = f["count"]
    return s


def evaluate(s: State, use_tree: bool = True) -> State:
    """Density stage then force stage (Section 2: two distinct stages)."""
    compute_density(s, use_tree)
    compute_force(s, use_tree=use_tree)
    return s


def wrap(x: np.ndarray, box: np.ndarray, box_offsets: np.ndarray) -> np.ndarray:
    out = x.copy()
    for b in range(box.shape[0]):
        sl = slice(int(box_offsets[b]), int(box_offsets[b + 1]))
        y = np.mod(out[sl], box[b])
        y[y >= box[b]] = 0.0
        out[sl] = y
    return out


def kdk_step(s: State, dt: float, use_tree: bool = True) -> State:
    """One kick-drift-kick step with a global time step dt.

    Requires a and du/dt of the current positions (call evaluate() first).
    Half kick of v and u, drift of x (periodic wrap), prediction of v and u
    to the end of the step for the new force evaluation (P_i uses the
    predicted u), density and force at the new positions, second half kick.
    """
    if s.a is None:
        raise ValueError("kdk_step needs a force evaluation of the current state")
    v_half = s.v + 0.5 * dt * s.a
    u_half = s.u + 0.5 * dt * s.dudt
    s.x = wrap(s.x + dt * v_half, s.box, s.box_offsets)
    v_pred = v_half + 0.5 * dt * s.a
    u_pred = u_half + 0.5 * dt * s.dudt
    if np.any(u_pred <= 0):
        raise OracleError(ENONPHYSICAL, "kdk_step (u <= 0)")
    compute_density(s, use_tree)
    compute_force(s, v=v_pred, u=u_pred, use_tree=use_tree)
    s.v = v_half + 0.5 * dt * s.a
    s.u = u_half + 0.5 * dt * s.dudt
    s.t += dt
    if np.any(s.u <= 0):
        raise OracleError(ENONPHYSICAL, "kdk_step (u <= 0)")
    return s


def diagnostics(s: State) -> dict:
    """Total momentum sum m v and total energy sum m (v^2 / 2 + u)."""
    return {"momentum": (s.m[:, None] * s.v).sum(axis=0),
            "energy": float((s.m * (0.5 * (s.v ** 2).sum(axis=1) + s.u)).sum())}
