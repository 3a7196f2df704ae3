"""The batched form's neighbour cache (reuse_lists = 2: on whatever the set's
size), through the C ABI and
against the FP64 oracle. The density stores each group's staged neighbours
and per-lane lists; the force of the same call takes its pairs from them
(plus the pairs a neighbour's larger h adds), and later density calls reuse
them while the summed |v dt| since they were built shows them complete.
Results must match the oracle and the uncached form whichever path a group
took: built, reused, rebuilt after particles moved too far, or sent to the
full force path by a particle of large h outside its stage."""
import numpy as np
import pytest

from paper_1606_02738_gb300 import inputs
from paper_1606_02738_gb300 import sph
from _parity import compare_density, compare_force, force_counts_close, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sph.lib()


FIELDS = ("x", "v", "u", "h", "rho", "omega", "P", "a", "dudt", "nngb", "nforce")


def _steps(p, n, dt, per_step=False, **kw):
    c = sph.Context(**kw).load(p)
    c.density()
    c.force()
    hist = [c.stats()]
    for _ in range(n):
        c.step(dt, 1)
        hist.append(c.stats())
    out = {k: c.get(k).cpu().numpy() for k in FIELDS}
    out["stats"] = hist[-1]
    out["hist"] = hist
    c.close()
    return out


@pytest.mark.parametrize("tile,precision", [(0, sph.SPH_PREC_FP32), (1, sph.SPH_PREC_FP32),
                                            (0, sph.SPH_PREC_KAHAN)],
                         ids=["tile0", "tile1", "kahan"])
def test_later_calls_reuse_density_and_force(tile, precision):
    """The first call (from the generator's uniform h guess, far from the
    clustered roots) builds every group's cache; later calls on the same
    positions and the converged h run most groups' density and force on it."""
    p = inputs.clustered(30011, n_spheres=8, seed=81, sigma_v=0.2)
    c = sph.Context(tile=tile, precision=precision, reuse_lists=2).load(p)
    c.density()
    c.force()
    st1 = c.stats()
    assert st1["cache_built_groups"] == st1["n_groups"] > 0
    assert st1["cache_density_groups"] == 0
    # groups whose stage overflowed from the uniform guess (clumps) stored
    # none; the second call stores theirs from the converged h
    c.density()
    c.force()
    c.density()
    c.force()
    st = c.stats()
    g = {k: c.get(k).cpu().numpy() for k in FIELDS}
    c.close()
    assert st["cache_density_groups"] > 0.5 * st["n_groups"], st["cache_density_groups"]
    # clumps put particles of large h beside most groups, which then take the
    # full force path (and the cached force is skipped while it would serve
    # fewer than an eighth of the groups); the results do not depend on it
    s = run_oracle(p)
    compare_density(g, s)
    compare_force(g, s)
    force_counts_close(g, s)


@pytest.mark.parametrize("tile,precision", [(0, sph.SPH_PREC_FP32), (1, sph.SPH_PREC_FP32),
                                            (0, sph.SPH_PREC_KAHAN)],
                         ids=["tile0", "tile1", "kahan"])
def test_sod_steps_reuse_the_cache_and_match_oracle(tile, precision):
    """Steps of a reduced shock tube: after the first call most groups run
    their density and force on the stored neighbours; results follow the
    oracle as closely as without the cache."""
    p = inputs.sod(nx_left=96, n_yz_left=24, nx_right=48, n_yz_right=12)
    dt, n = 2e-3, 6
    g = _steps(p, n, dt, tile=tile, precision=precision, reuse_lists=2)
    last = g["stats"]
    assert last["cache_density_groups"] > 0.5 * last["n_groups"], last["cache_density_groups"]
    assert last["cache_force_groups"] > 0.5 * last["n_groups"], last["cache_force_groups"]
    s = run_oracle(p, steps=n, dt=dt)
    compare_density(g, s, tol_rho=2e-5, tol_h=2e-5, counts=False, check_P=False)
    compare_force(g, s, tol_a=3e-4, tol_du=3e-4)
    g0 = _steps(p, n, dt, tile=tile, precision=precision, reuse_lists=0)
    assert g0["stats"]["cache_built_groups"] == 0 and g0["stats"]["cache_force_groups"] == 0
    # the two forms sum in different orders: forces within 1e-4 max|a| of each
    # other move x apart by at most n^2 dt^2 1e-4 max|a|
    amax = np.abs(g0["a"]).max()
    np.testing.assert_allclose(g["x"], g0["x"], rtol=0, atol=n * n * dt * dt * 1e-4 * amax)
    assert np.max(np.abs(g["h"] / g0["h"] - 1)) < 5e-6
    assert np.max(np.abs(g["rho"] / g0["rho"] - 1)) < 5e-6
    assert np.abs(g["a"] - g0["a"]).max() < 1e-4 * np.abs(g0["a"]).max()


def test_fast_motion_rebuilds_groups_and_still_matches_oracle():
    """Random velocities of ~2.6 with steps moving particles by ~4% of h:
    stored neighbours stop covering their h within a couple of steps, groups
    rebuild (and an epoch restarts), results stay on the oracle's."""
    p = inputs.uniform(20000, seed=403, sigma_v=1.5)
    p.u = np.full(p.n, 10.0, dtype=np.float32)  # sound speed 3.3: a subsonic flow
    dt, n = 1.5e-3, 6
    g = _steps(p, n, dt, reuse_lists=2)
    built_later = sum(h["cache_built_groups"] for h in g["hist"][2:])
    assert built_later > 0, [h["cache_built_groups"] for h in g["hist"]]
    s = run_oracle(p, steps=n, dt=dt)
    compare_density(g, s, tol_rho=2e-5, tol_h=2e-5, counts=False, check_P=False)
    compare_force(g, s, tol_a=3e-4, tol_du=3e-4)


def test_large_h_next_to_small_h_takes_the_full_force_path():
    """A lattice of spacing a (x < 2/3) beside one of spacing 3a: the coarse
    particles' h (about 6.8 a) reaches deep into the fine region from beyond
    the fine groups' stages, so the fine groups near the two interfaces take
    the full force path while those in the middle run on the cache (second
    call, converged h); results match the oracle element by element."""
    n = 36
    a = 1.0 / n
    fx = (np.arange(24) + 0.5) * a
    f1 = (np.arange(n) + 0.5) * a
    fine = np.stack(np.meshgrid(fx, f1, f1, indexing="ij"), -1).reshape(-1, 3)
    cx = 2.0 / 3.0 + (np.arange(4) + 0.5) * 3 * a
    c1 = (np.arange(n // 3) + 0.5) * 3 * a
    coarse = np.stack(np.meshgrid(cx, c1, c1, indexing="ij"), -1).reshape(-1, 3)
    x = np.concatenate([fine, coarse])
    rng = np.random.default_rng(9)
    x = x + rng.uniform(-0.01 * a, 0.01 * a, x.shape)
    p = inputs.uniform(x.shape[0], seed=404, sigma_v=0.2)
    p.x = np.mod(x, 1.0)
    p.h = np.full(p.n, 2.5 * a)
    c = sph.Context(reuse_lists=2).load(p)
    c.density()
    c.force()
    c.density()
    c.force()
    st = c.stats()
    g = {k: c.get(k).cpu().numpy() for k in FIELDS}
    c.close()
    assert 0 < st["cache_force_groups"] < st["n_groups"], (st["cache_force_groups"],
                                                           st["n_groups"])
    s = run_oracle(p)
    compare_density(g, s)
    compare_force(g, s)
    force_counts_close(g, s)
