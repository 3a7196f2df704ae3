"""Bit-exact integer cell indices (Section 3.1: particles are binned into
cells no smaller than the largest smoothing length, then cells are split
recursively). The library's top-cell index of every particle must be
floor(x / w) exactly for the FP64 position x and the FP64 cell width w, and
its octree leaf cell must be the leading `level` bits of the 10-bit
sub-cell coordinate floor((x - c w) (1024 / w)). The reference here uses
exact rational arithmetic (fractions.Fraction), so it owes nothing to
floating-point rounding of x / w; the cases put particles exactly on cell
faces, one ulp on either side of them, at 0, at the largest double below
the box edge, and on the positions after drift steps with and without
regrids."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1606_02738_gb300 import inputs
from paper_1606_02738_gb300 import sph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sph.lib()


def _exact_cells(x, n, w):
    """Top-cell coordinates and 10-bit sub-cell coordinates, exactly."""
    top = np.zeros(x.shape, dtype=np.int64)
    sub = np.zeros(x.shape, dtype=np.int64)
    for d in range(3):
        wd = Fraction(w[d])
        iw1024 = (1.0 / w[d]) * 1024.0  # (1 / w) rounded once, times a power of two
        for k in range(x.shape[0]):
            xf = Fraction(float(x[k, d]))
            c = math.floor(xf / wd)
            c = min(max(c, 0), n[d] - 1)
            rel = float(xf - c * wd)     # x - c w, rounded once
            q = math.floor(rel * iw1024)
            top[k, d] = c
            sub[k, d] = min(max(q, 0), 1023)
    return top, sub


def _check(c, x):
    g = c.grid(0)
    top, sub = _exact_cells(x, g["n"], g["w"])
    cell = c.get("cell").cpu().numpy().astype(np.int64)
    leaf = c.get("leaf_cell").cpu().numpy().astype(np.int64)
    assert np.array_equal(cell[:, :3], top), np.argwhere(cell[:, :3] != top)[:5]
    level = cell[:, 3]
    assert level.min() >= 0 and level.max() <= 10
    assert np.array_equal(leaf, sub >> (10 - level)[:, None])
    return g


def _face_set(seed):
    """A uniform set (cells of edge >= h_max, about 11 per axis) with 1,800
    particles moved so that one coordinate lies on a cell face, one ulp
    above one, or one ulp below one, and three at the box corner 0 and at the
    last double below the edge L = 1."""
    p = inputs.uniform(30000, seed=seed, sigma_v=0.3)
    c = sph.Context(cell_factor=1.0).load(p)
    g = c.grid(0)
    c.close()
    rng = np.random.default_rng(seed)
    x = np.array(p.x)
    w = np.asarray(g["w"])
    for d in range(3):
        for kind in range(3):
            rows = slice(600 * d + 200 * kind, 600 * d + 200 * (kind + 1))
            on = rng.integers(0, g["n"][d], 200) * w[d]   # on a face (the rounded product)
            if kind == 1:
                on = np.nextafter(on, np.inf)              # one ulp above
            elif kind == 2:
                on = np.nextafter(np.maximum(on, 1e-300), -np.inf)  # one ulp below
            x[rows, d] = on
    x[1800, :] = 0.0
    x[1801, :] = np.nextafter(1.0, 0.0)          # 1 - 2^-53, the last double below L = 1
    x[1802, :] = [1.0 - 1e-16, 0.5, 0.25]        # 1 - 1e-16 rounds to the same double
    p.x = x
    return p


def test_cells_exact_on_faces_and_box_edges():
    p = _face_set(inputs.SEED_BASE + 41)
    c = sph.Context(cell_factor=1.0).load(p)
    xw = c.get("x").cpu().numpy()
    assert np.array_equal(xw, p.x)  # already inside [0, L): loaded unchanged
    _check(c, xw)
    c.close()


def test_cells_exact_after_drift_with_and_without_regrid():
    p = _face_set(inputs.SEED_BASE + 42)
    # regrid every step: the cells are those of the drifted positions
    c = sph.Context(reuse_grid=False, cell_factor=1.0).load(p)
    c.density()
    c.force()
    c.step(2e-3, 2)
    _check(c, c.get("x").cpu().numpy())
    c.close()
    # reused grid: the cells stay those of the positions at the last regrid
    # (a step regrids unless the grid of the previous one is known to reach)
    c = sph.Context(reuse_grid=True, cell_factor=1.0).load(p)
    c.density()
    c.force()
    x_regrid = c.get("x").cpu().numpy()
    reused = redone = 0
    for _ in range(3):
        c.step(2e-3, 1)
        st = c.stats()
        if st["reused_steps"] == reused or st["redone_steps"] > redone:  # a regrid
            x_regrid = c.get("x").cpu().numpy()
        reused, redone = st["reused_steps"], st["redone_steps"]
    assert reused - redone >= 1
    _check(c, x_regrid)
    c.close()
