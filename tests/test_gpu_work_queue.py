"""The batched first tier's work queue (Section 3.2, task queue and task
costs): the first-tier kernels claim their target groups 32 at a time from
a device queue, in group order (work_queue = 2) or in the order of the
costs measured in the previous call (work_queue = 3), instead of a fixed
grid stride (work_queue = 0). Groups are independent, so every result must
be bit-identical in every mode, on every path a group can take (first,
second and third tiers, the neighbour cache's split of the first tier),
over steps whose cost order comes from the costs measured in the step
before; and the queued run must match the FP64 oracle."""
import numpy as np
import pytest

from paper_1606_02738_gb300 import inputs
from paper_1606_02738_gb300 import sph
from _parity import compare_density, compare_force, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sph.lib()


FIELDS = ("x", "v", "u", "h", "rho", "omega", "P", "a", "dudt", "nngb", "nforce")


def _run(p, steps, dt, **kw):
    c = sph.Context(**kw).load(p)
    c.density()
    c.force()
    for _ in range(steps):
        c.step(dt, 1)
    out = {k: c.get(k).cpu().numpy() for k in FIELDS}
    out["stats"] = c.stats()
    c.close()
    return out


CASES = [
    # perturbed lattice: every group in the first tier
    ("uniform", lambda: inputs.config(1), dict(tile=0), 3e-3),
    # clustered, 20x h spread, moving: second and third tiers are used
    ("clustered", lambda: inputs.clustered(60_000, seed=5, sigma_v=0.2),
     dict(tile=1, n_split=32), 1e-4),
    # lognormal with the neighbour cache forced on (two first-tier launches
    # share the queue's groups; the force skips the groups done on the cache)
    ("lognormal_cache", lambda: inputs.config(5, 0.004), dict(tile=1, reuse_lists=2), 2e-5),
]


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("name,make,kw,dt", CASES, ids=[c[0] for c in CASES])
def test_work_queue_is_bit_identical(name, make, kw, dt, mode):
    p = make()
    on = _run(p, 3, dt, work_queue=mode, **kw)
    off = _run(p, 3, dt, work_queue=0, **kw)
    for k in FIELDS:
        assert np.array_equal(on[k], off[k]), k
    for k in ("density_interactions", "force_interactions", "tier2_groups", "tier3_entries"):
        assert on["stats"][k] == off["stats"][k], k


def test_cost_ordered_queue_matches_oracle_on_clustered_set():
    p = inputs.clustered(40_000, seed=11)
    g = run_gpu(p, n_split=32, tile=1, work_queue=3)
    o = run_oracle(p)
    compare_density(g, o)
    compare_force(g, o)
