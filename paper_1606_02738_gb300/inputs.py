"""Seeded synthetic particle sets shaped like the paper's test problems.

The paper's own workloads are resampled EAGLE snapshots (Section 4.1), which
are not available here. These generators stand in for them with particle sets
of the same character: uniform gas, a shock-tube lattice, Plummer clusters that
make the smoothing length span about two decades, many independent boxes of
mixed size, and a lognormal density field.

This module holds no SPH arithmetic: it only draws positions, velocities,
masses, internal energies and an initial smoothing-length guess from seeded
NumPy generators. Both the FP64 oracle and the CUDA path consume exactly these
arrays (velocities, masses and internal energies are rounded to float32 once,
here, so both sides see the same values).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 160602738
GAMMA = 5.0 / 3.0
N_NGB = 48.0


@dataclass
class ParticleSet:
    """Particles of one or more independent periodic boxes.

    x: (N, 3) float64 positions wrapped into [0, L) of their box.
    v: (N, 3) float32 velocities.
    m, u: (N,) float32 masses and specific internal energies.
    h: (N,) float64 initial smoothing-length guesses (any positive value; the
       h iteration finds the unique root from it).
    box: (n_boxes, 3) float64 box edge lengths.
    box_offsets: (n_boxes + 1,) int64 particle ranges of the boxes.
    """

    name: str
    x: np.ndarray
    v: np.ndarray
    m: np.ndarray
    u: np.ndarray
    h: np.ndarray
    box: np.ndarray
    box_offsets: np.ndarray
    gamma: float = GAMMA
    n_ngb: float = N_NGB
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_boxes(self) -> int:
        return int(self.box.shape[0])

    def box_slice(self, b: int) -> slice:
        return slice(int(self.box_offsets[b]), int(self.box_offsets[b + 1]))

    def subset_box(self, b: int) -> "ParticleSet":
        return self.subset_boxes(b, b + 1, name=f"{self.name}[box {b}]")

    def subset_boxes(self, b0: int, b1: int, name: str | None = None) -> "ParticleSet":
        """Boxes b0 .. b1-1 as a set of their own (the boxes never interact)."""
        lo, hi = int(self.box_offsets[b0]), int(self.box_offsets[b1])
        return ParticleSet(
            name=name or f"{self.name}[boxes {b0}:{b1}]", x=self.x[lo:hi].copy(),
            v=self.v[lo:hi].copy(), m=self.m[lo:hi].copy(), u=self.u[lo:hi].copy(),
            h=self.h[lo:hi].copy(), box=self.box[b0:b1].copy(),
            box_offsets=(self.box_offsets[b0:b1 + 1] - lo).astype(np.int64),
            gamma=self.gamma, n_ngb=self.n_ngb, meta=dict(self.meta))


def h_guess_uniform(n_particles: int, volume: float = 1.0, factor: float = 1.2) -> float:
    """Initial guess 1.2 * (48 / (4/3 pi n))^(1/3) for n particles in `volume`."""
    n_density = n_particles / volume
    return factor * (N_NGB / (4.0 / 3.0 * np.pi * n_density)) ** (1.0 / 3.0)


def _wrap(x: np.ndarray, box: np.ndarray) -> np.ndarray:
    x = np.mod(x, box)
    # np.mod can return exactly box for tiny negative inputs; fold those to 0.
    x[x >= box] = 0.0
    return x


def _single(name, x, v, m, u, h, box, **meta) -> ParticleSet:
    box = np.asarray(box, dtype=np.float64).reshape(1, 3)
    x = _wrap(np.asarray(x, dtype=np.float64), box[0])
    n = x.shape[0]
    return ParticleSet(
        name=name, x=np.ascontiguousarray(x),
        v=np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(n, 3)),
        m=np.ascontiguousarray(np.broadcast_to(np.asarray(m, dtype=np.float32), (n,))),
        u=np.ascontiguousarray(np.broadcast_to(np.asarray(u, dtype=np.float32), (n,))),
        h=np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))),
        box=box, box_offsets=np.array([0, n], dtype=np.int64), meta=meta)


def uniform(n: int = 32768, seed: int = SEED_BASE + 1, sigma_v: float = 0.0,
            box=(1.0, 1.0, 1.0), name: str = "uniform") -> ParticleSet:
    """Uniform random gas in a periodic box: m = M/N with M = box volume,
    u = 1, v = 0 (or N(0, sigma_v) per component), h from the uniform guess."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    x = rng.random((n, 3)) * box
    v = rng.normal(0.0, sigma_v, (n, 3)) if sigma_v > 0 else np.zeros((n, 3))
    vol = float(np.prod(box))
    return _single(name, x, v, vol / n, 1.0, h_guess_uniform(n, vol), box,
                   seed=seed, sigma_v=sigma_v)


def lattice(n_side: int = 12, jitter: float = 0.0, seed: int = SEED_BASE + 11,
            box_len: float = 1.0, sigma_v: float = 0.0, h_factor: float = 2.4,
            name: str = "lattice") -> ParticleSet:
    """Simple-cubic lattice of n_side^3 particles, spacing a = L / n_side,
    optionally jittered by +-jitter*a per axis, equal masses with mean
    density 1. Initial h = h_factor * a."""
    rng = np.random.default_rng(seed)
    a = box_len / n_side
    g = (np.arange(n_side) + 0.5) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if jitter > 0:
        x = x + rng.uniform(-jitter * a, jitter * a, x.shape)
    n = x.shape[0]
    v = rng.normal(0.0, sigma_v, (n, 3)) if sigma_v > 0 else np.zeros((n, 3))
    return _single(name, x, v, box_len ** 3 / n, 1.0, h_factor * a, [box_len] * 3,
                   spacing=a, seed=seed)


def sod(nx_left: int = 240, n_yz_left: int = 60, nx_right: int = 120,
        n_yz_right: int = 30, jitter: float = 0.01, seed: int = SEED_BASE + 2,
        name: str = "sod") -> ParticleSet:
    """3D Sod shock tube in the periodic box [0,2] x [0,0.25]^2.

    Left half x < 1: cubic lattice of spacing 1/240 with rho = 1, P = 1;
    right half: cubic lattice of spacing 1/120 with rho = 0.125, P = 0.1.
    Equal particle masses (the 8:1 density contrast is an 8:1 contrast in
    number density, i.e. a 2:1 lattice-spacing ratio). Each particle is
    jittered uniformly by +-jitter * a per axis. u = P / ((gamma-1) rho):
    1.5 on the left, 1.2 on the right. v = 0.
    """
    rng = np.random.default_rng(seed)
    box = np.array([2.0, 0.25, 0.25])

    def block(nx, nyz, x0):
        a = 1.0 / nx
        gx = x0 + (np.arange(nx) + 0.5) * a
        gyz = (np.arange(nyz) + 0.5) * (0.25 / nyz)
        p = np.stack(np.meshgrid(gx, gyz, gyz, indexing="ij"), -1).reshape(-1, 3)
        return p + rng.uniform(-jitter * a, jitter * a, p.shape), a

    xl, al = block(nx_left, n_yz_left, 0.0)
    xr, ar = block(nx_right, n_yz_right, 1.0)
    x = np.concatenate([xl, xr])
    m = 1.0 * 1.0 * 0.25 * 0.25 / xl.shape[0]
    g = GAMMA
    u = np.concatenate([np.full(xl.shape[0], 1.0 / ((g - 1) * 1.0)),
                        np.full(xr.shape[0], 0.1 / ((g - 1) * 0.125))])
    # local uniform-density guess per side
    h = np.concatenate([np.full(xl.shape[0], h_guess_uniform(1, al ** 3)),
                        np.full(xr.shape[0], h_guess_uniform(1, ar ** 3))])
    return _single(name, x, np.zeros_like(x), m, u, h, box, seed=seed,
                   n_left=xl.shape[0], n_right=xr.shape[0])


def _plummer_positions(rng, n_per, centres, radii, r_max=0.5):
    """Draw n_per points around each centre from a Plummer profile with scale
    radius a: r = a / sqrt(X^(-2/3) - 1), X ~ U(0,1), rejecting r > r_max;
    isotropic directions."""
    out = []
    for c, a in zip(centres, radii):
        r = np.empty(0)
        while r.size < n_per:
            X = rng.random(2 * n_per)
            X = X[X > 0]
            rr = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
            r = np.concatenate([r, rr[rr <= r_max]])
        r = r[:n_per]
        d = rng.normal(size=(n_per, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        out.append(c + r[:, None] * d)
    return np.concatenate(out)


def clustered(n: int = 4194304, n_spheres: int = 64, frac_clustered: float = 0.7,
              a_min: float = 0.005, a_max: float = 0.05, seed: int = SEED_BASE + 3,
              sigma_v: float = 0.0, name: str = "clustered") -> ParticleSet:
    """Plummer spheres (equal particle counts, scale radii log-uniform in
    [a_min, a_max], centres uniform) holding frac_clustered of the particles,
    plus a uniform background, in the periodic unit box. m = 1/N, u = 1."""
    rng = np.random.default_rng(seed)
    n_per = int(round(frac_clustered * n / n_spheres))
    n_bg = n - n_per * n_spheres
    centres = rng.random((n_spheres, 3))
    radii = np.exp(rng.uniform(np.log(a_min), np.log(a_max), n_spheres))
    xc = _plummer_positions(rng, n_per, centres, radii)
    xb = rng.random((n_bg, 3))
    x = np.concatenate([xc, xb])
    v = rng.normal(0.0, sigma_v, (n, 3)) if sigma_v > 0 else np.zeros((n, 3))
    return _single(name, x, v, 1.0 / n, 1.0, h_guess_uniform(n), [1.0] * 3,
                   seed=seed, n_spheres=n_spheres, radii=radii.tolist())


def batched(n_boxes: int = 256, n_min: int = 1024, n_max: int = 262144,
            seed: int = SEED_BASE + 4, name: str = "batched",
            min_clustered: int = 4096) -> ParticleSet:
    """Independent periodic unit boxes; box b holds
    N_b = round(exp(U(ln n_min, ln n_max))) particles, uniform random with
    probability 1/2, else the clustered generator with 8 Plummer spheres
    scaled to N_b. m = 1/N_b, u = 1, v = 0.

    A clustered box needs at least `min_clustered` particles: below that its
    uniform 30% background is too sparse for 48 neighbours within L/3 (the
    largest smoothing length a periodic box of three cells per axis admits),
    so such boxes are uniform."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_boxes))).astype(np.int64)
    kinds = rng.random(n_boxes) < 0.5
    parts = []
    for b in range(n_boxes):
        s = int(rng.integers(0, 2**31 - 1))
        if kinds[b] or sizes[b] < min_clustered:
            p = uniform(int(sizes[b]), seed=s)
        else:
            p = clustered(int(sizes[b]), n_spheres=8, seed=s)
        parts.append(p)
    offs = np.zeros(n_boxes + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    return ParticleSet(
        name=name,
        x=np.ascontiguousarray(np.concatenate([p.x for p in parts])),
        v=np.ascontiguousarray(np.concatenate([p.v for p in parts])),
        m=np.ascontiguousarray(np.concatenate([p.m for p in parts])),
        u=np.ascontiguousarray(np.concatenate([p.u for p in parts])),
        h=np.ascontiguousarray(np.concatenate([p.h for p in parts])),
        box=np.ones((n_boxes, 3)), box_offsets=offs,
        meta={"seed": seed, "sizes": sizes.tolist(), "uniform": kinds.tolist()})


def lognormal(n: int = 1 << 26, grid: int = 256, sigma_lnrho: float = 1.5,
              seed: int = SEED_BASE + 5, sigma_v: float = 0.1, sigma_lnu: float = 0.5,
              name: str = "lognormal") -> ParticleSet:
    """Poisson sample of a lognormal density field in the periodic unit box.

    g: Gaussian random field on grid^3 (white noise times sqrt(P(k)),
    P(k) ~ k^-2, k = 0 mode zeroed), normalised to unit variance;
    ln rho = sigma g - sigma^2 / 2. The n particles are spread over the grid
    cells by one multinomial draw with probabilities rho_c / sum(rho), and
    placed uniformly inside their cell. v ~ N(0, sigma_v) per component,
    ln u ~ N(0, sigma_lnu^2), m = 1/n.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((grid, grid, grid))
    k = np.fft.fftfreq(grid) * grid
    kz = np.fft.rfftfreq(grid) * grid
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = 1.0 / np.sqrt(k2[nz])          # sqrt(P(k)) with P ~ k^-2
    g = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=noise.shape)
    del noise
    g = (g - g.mean()) / g.std()
    rho = np.exp(sigma_lnrho * g - 0.5 * sigma_lnrho ** 2).ravel()
    del g
    counts = rng.multinomial(n, rho / rho.sum())
    del rho
    cell = np.repeat(np.arange(grid ** 3, dtype=np.int64), counts)
    del counts
    ix = cell // (grid * grid)
    iy = (cell // grid) % grid
    iz = cell % grid
    del cell
    x = np.empty((n, 3))
    x[:, 0] = ix
    x[:, 1] = iy
    x[:, 2] = iz
    del ix, iy, iz
    x += rng.random((n, 3))
    x /= grid
    v = rng.normal(0.0, sigma_v, (n, 3)).astype(np.float32)
    u = np.exp(rng.normal(0.0, sigma_lnu, n)).astype(np.float32)
    return _single(name, x, v, 1.0 / n, u, h_guess_uniform(n), [1.0] * 3,
                   seed=seed, grid=grid, sigma_lnrho=sigma_lnrho)


def config(k: int, scale: float = 1.0) -> ParticleSet:
    """The five workloads, k = 1..5. `scale` < 1 shrinks the particle count
    (same recipe, same seed) for tests that need a quicker oracle."""
    if k == 1:
        return uniform(max(64, int(round(32768 * scale))), seed=SEED_BASE + 1, name="cfg1_uniform")
    if k == 2:
        if scale >= 1.0:
            return sod(name="cfg2_sod")
        f = scale ** (1.0 / 3.0)
        nl = max(8, int(round(240 * f)) // 4 * 4)
        return sod(nx_left=nl, n_yz_left=nl // 4, nx_right=nl // 2, n_yz_right=nl // 8,
                   name="cfg2_sod_small")
    if k == 3:
        return clustered(max(4096, int(round(4194304 * scale))), name="cfg3_clustered")
    if k == 4:
        if scale >= 1.0:
            return batched(name="cfg4_batched")
        nb = max(2, int(round(256 * scale ** 0.5)))
        return batched(n_boxes=nb, n_min=256, n_max=max(1024, int(262144 * scale ** 0.5)),
                       name="cfg4_batched_small")
    if k == 5:
        if scale >= 1.0:
            return lognormal(name="cfg5_lognormal")
        grid = max(16, int(round(256 * scale ** (1.0 / 3.0))))
        return lognormal(n=max(4096, int(round((1 << 26) * scale))), grid=grid,
                         name="cfg5_lognormal_small")
    raise ValueError(f"unknown config {k}")
