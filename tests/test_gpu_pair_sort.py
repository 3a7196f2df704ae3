"""Pair-axis sorts (Section 3.1: the particles of every cell are sorted along
the axes joining it to its neighbours before the density tasks) and the
pruning they allow, through the C ABI.

The sort itself is checked against its definition: along each of the 13
directions e_k every leaf's particles appear in order of x . e_k (computed
here in FP64 from the caller's positions), each particle exactly once. Where
two keys are closer than the FP32 resolution of the leaf-relative positions
either order is correct, so the test allows inversions only that small.

The pruning must not change what is computed: the per-pass form with and
without sorts matches the oracle, the two agree with each other, and the
pruned form tests fewer pairs.
"""
import numpy as np
import pytest

from paper_1606_02738_gb300 import inputs
from paper_1606_02738_gb300 import sph
from _parity import (TOL_RHO, compare_density, compare_force, edge_pairs, force_counts_close,
                     run_gpu, run_oracle)

pytestmark = pytest.mark.gpu

AXES = np.array([(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1),
                 (0, 1, 1), (0, 1, -1), (1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1)],
                dtype=np.float64)
AXES /= np.linalg.norm(AXES, axis=1, keepdims=True)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sph.lib()


def _check_orders(p, c):
    n = p.n
    leaf0 = None
    members0 = None
    for k in range(13):
        order, leaf = (t.cpu().numpy().astype(np.int64) for t in c.pair_order(k))
        assert np.array_equal(np.sort(order), np.arange(n)), "not a permutation"
        assert np.all(np.diff(leaf) >= 0), "leaves must occupy consecutive slots"
        if leaf0 is None:
            leaf0 = leaf
        assert np.array_equal(leaf, leaf0), "leaf layout differs between axes"
        starts = np.flatnonzero(np.r_[True, leaf[1:] != leaf[:-1]])
        ends = np.r_[starts[1:], n]
        members = [np.sort(order[a:b]) for a, b in zip(starts, ends)]
        if members0 is None:
            members0 = members
        for m, m0 in zip(members, members0):
            assert np.array_equal(m, m0), "a leaf holds different particles on another axis"
        # keys in FP64 from caller positions, each taken at the periodic image
        # nearest the first particle of its leaf (after steps on a reused grid
        # a leaf's particles may straddle the box boundary)
        box_of = np.searchsorted(p.box_offsets, order, side="right") - 1
        L = p.box[box_of]
        x = p.x[order]
        first = x[starts[np.searchsorted(starts, np.arange(n), side="right") - 1]]
        d = x - first
        d -= L * np.round(d / L)
        key = (first + d) @ AXES[k]
        tol = 2e-6 * L.max(axis=1)
        step = np.diff(key)
        same_leaf = leaf[1:] == leaf[:-1]
        bad = same_leaf & (step < -tol[1:])
        assert not bad.any(), (k, int(bad.sum()), float(step[bad].min()))
    return len(members0)


def test_pair_orders_uniform_ragged_leaves():
    p = inputs.uniform(6007, seed=301, sigma_v=0.2)
    c = sph.Context(n_split=17).load(p)
    n_leaves = _check_orders(p, c)
    assert n_leaves == c.stats()["n_leaves"] and n_leaves > 100
    c.close()


def test_pair_orders_clustered_and_after_steps():
    p = inputs.clustered(8192, seed=302, sigma_v=0.1)
    c = sph.Context().load(p)
    _check_orders(p, c)
    c.density()
    c.force()
    c.step(1e-3, 3)
    # the sorts follow the regrid of every step: check against the drifted x
    x = c.get("x").cpu().numpy()
    q = inputs.ParticleSet(name=p.name, x=x, v=p.v, m=p.m, u=p.u, h=p.h, box=p.box,
                           box_offsets=p.box_offsets)
    _check_orders(q, c)
    c.close()


def test_pair_orders_batched_boxes():
    p = inputs.batched(6, n_min=2000, n_max=5000, seed=303)
    c = sph.Context().load(p)
    _check_orders(p, c)
    c.close()


def test_pair_order_errors():
    p = inputs.uniform(2000, seed=304)
    c = sph.Context(pair_sort=False).load(p)
    with pytest.raises(sph.SphError) as e:
        c.pair_order(0)
    assert e.value.code == sph.SPH_ESTATE
    c.close()
    c = sph.Context().load(p)
    with pytest.raises(sph.SphError) as e:
        c.pair_order(13)
    assert e.value.code == sph.SPH_EINVAL
    c.close()


@pytest.mark.parametrize("make", [
    lambda: inputs.uniform(6007, seed=311, sigma_v=0.3),
    lambda: inputs.clustered(8192, seed=312, sigma_v=0.2),
    lambda: inputs.sod(nx_left=96, n_yz_left=24, nx_right=48, n_yz_right=12),
], ids=["uniform", "clustered", "sod"])
def test_pruned_per_pass_form_matches_unpruned_and_oracle(make):
    p = make()
    s = run_oracle(p)
    g1 = run_gpu(p, mode=sph.SPH_MODE_PLAIN, pair_sort=True)
    g0 = run_gpu(p, mode=sph.SPH_MODE_PLAIN, pair_sort=False)
    for g in (g0, g1):
        compare_density(g, s)
        compare_force(g, s)
        force_counts_close(g, s)
    # the two runs sum in different orders, so their converged h differ in the
    # last FP32 bits: counts may differ only by pairs within 1e-6 h of an edge
    amb = edge_pairs(s)
    assert np.all(np.abs(g1["nngb"].astype(np.int64) - g0["nngb"]) <= amb)
    np.testing.assert_allclose(g1["rho"], g0["rho"], rtol=2 * TOL_RHO)
    s0, s1 = g0["stats"], g1["stats"]
    assert s1["density_interactions"] == pytest.approx(s0["density_interactions"], rel=1e-5)
    assert s1["force_interactions"] == pytest.approx(s0["force_interactions"], rel=1e-5)
    assert s1["density_pair_candidates"] < s0["density_pair_candidates"]
    assert s1["force_pair_candidates"] < s0["force_pair_candidates"]


@pytest.mark.parametrize("tile", [0, 1])
def test_batched_direct_modes_match_oracle(tile):
    """Large neighbour numbers overflow the batched kernels' per-lane lists
    (n_ngb >= 120) and the force kernel's per-warp candidate lists (around
    n_ngb = 160-200, while its stage still fits). With tile 0 those warps read
    their candidates, or the whole stage, directly; with tile 1 the density
    does the same and the force works through its candidates in chunks and
    its lists in rounds. Every form must give the oracle's results."""
    direct = np.zeros(2, dtype=np.int64)
    for n_ngb in (120.0, 160.0, 200.0):
        p = inputs.uniform(12000, seed=321, sigma_v=0.2)
        p.n_ngb = n_ngb
        g = run_gpu(p, mode=sph.SPH_MODE_BATCHED, n_ngb=n_ngb, tile=tile)
        s = run_oracle(p)
        compare_density(g, s)
        compare_force(g, s)
        direct += [g["stats"]["direct_list_warps"], g["stats"]["direct_stage_warps"]]
    assert direct[0] > 0 and direct[1] > 0, direct
