"""The batched form's three tiers on inputs that need them, through the C ABI
and against the FP64 oracle.

Tier 1 stages a group of <= 32 particles by its bounding box; a group whose
stage overflows is staged again by each target's own radius (tier 2); a
group that overflows that too, or its task slots, or whose h outgrows the
staged radius, is computed one warp per target by a direct walk of the
octrees (tier 3). Large h contrast (dense clumps beside sparse background)
and very large neighbour numbers drive particles into tiers 2 and 3; the
results must still match the oracle, and nothing may be left to the
per-pass form.
"""
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


@pytest.mark.parametrize("precision,tile", [(sph.SPH_PREC_FP32, 0), (sph.SPH_PREC_KAHAN, 0),
                                            (sph.SPH_PREC_KAHAN, 1)])
def test_clustered_from_flat_guess_uses_tiers_2_and_3(precision, tile):
    """A uniform initial h over strong clumps: the first density pushes many
    groups past their stage (their h shrinks or grows far from the guess)."""
    p = inputs.clustered(60000, n_spheres=8, seed=11, sigma_v=0.1)
    g = run_gpu(p, mode=sph.SPH_MODE_BATCHED, precision=precision, tile=tile)
    s = run_oracle(p)
    assert s.h.max() / s.h.min() > 20
    st = g["stats"]
    assert st["tier2_groups"][0] > 0 and st["tier3_entries"][0] > 0, st
    assert st["batched_fallbacks"] == 0, st
    compare_density(g, s)
    compare_force(g, s)
    force_counts_close(g, s)


@pytest.mark.parametrize("tile", [0, 2])
def test_clustered_steady_state_second_call(tile):
    """At converged h (second density + force on the same state) the tiers
    still give the oracle's values; with tile 2 the second force call runs
    the first tier in two parts, the small stage for the groups whose first
    call's stage fitted it and the large one for the rest."""
    p = inputs.clustered(60000, n_spheres=8, seed=12, sigma_v=0.1)
    c = sph.Context(mode=sph.SPH_MODE_BATCHED, tile=tile).load(p)
    c.density()
    c.force()
    c.density()
    c.force()
    st = c.stats()
    g = {k: c.get(k).cpu().numpy() for k in ("h", "rho", "omega", "P", "a", "dudt", "nngb",
                                              "nforce")}
    c.close()
    s = run_oracle(p)
    assert st["batched_fallbacks"] == 0, st
    assert st["tier2_groups"][0] + st["tier2_groups"][1] > 0, st
    compare_density(g, s)
    compare_force(g, s)


def test_huge_neighbour_number_reaches_tier_3_for_density_and_force():
    """n_ngb = 2000: the union of a group's 32 spheres holds more particles
    than the second tier's stage, for the density and for the force."""
    p = inputs.uniform(40000, seed=331, sigma_v=0.2)
    p.n_ngb = 2000.0
    g = run_gpu(p, mode=sph.SPH_MODE_BATCHED, n_ngb=2000.0)
    s = run_oracle(p)
    st = g["stats"]
    assert st["tier3_entries"][0] > 0 and st["tier3_entries"][1] > 0, st
    assert st["batched_fallbacks"] == 0, st
    compare_density(g, s)
    compare_force(g, s)


def test_boxes_in_one_context_match_one_context_per_box():
    """Independent periodic boxes in one context (one launch sequence for all)
    give each box the results it gets alone: the boxes never interact."""
    p = inputs.batched(n_boxes=5, n_min=2000, n_max=8000, seed=77)
    p.v = p.v.copy()
    for k in range(5):
        p.v[p.box_slice(k)] += np.float32(0.1 * k)  # a different bulk motion per box
    g = run_gpu(p, steps=2, dt=1e-3, mode=sph.SPH_MODE_BATCHED)
    for b in range(p.n_boxes):
        q = p.subset_box(b)
        gb = run_gpu(q, steps=2, dt=1e-3, mode=sph.SPH_MODE_BATCHED)
        sl = p.box_slice(b)
        np.testing.assert_allclose(g["x"][sl], gb["x"], rtol=0, atol=1e-9)
        assert np.max(np.abs(g["rho"][sl] / gb["rho"] - 1)) < 5e-6
        assert np.abs(g["a"][sl] - gb["a"]).max() < 5e-5 * np.abs(gb["a"]).max()
