"""The allocation-free density entry point (sph_density_noalloc) against the
regular one (sph_init + sph_density + sph_get), through the C ABI.

sph_density_noalloc exists for callers that may not allocate device memory
on their calls (a framework that owns the GPU through its own pool, or code
where cudaMalloc/cudaFree is not allowed); it keeps its scratch in a fixed
device array shared by all calls. Two calls in a row on different particle
sets must each match the regular path, so nothing left in the scratch by the
first call leaks into the second. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1606_02738_gb300 import inputs
from paper_1606_02738_gb300 import sph

pytestmark = pytest.mark.gpu

TOL_H = 1e-5
TOL_RHO = 1e-5
TOL_OMEGA = 1e-4


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _regular(p):
    c = sph.Context().load(p)
    c.density()
    out = {k: c.get(k).cpu().numpy() for k in ("h", "rho", "omega")}
    c.close()
    return out


def _noalloc(torch, p):
    dev = torch.device("cuda")
    x = torch.as_tensor(np.array(p.x), dtype=torch.float64, device=dev)
    m = torch.as_tensor(np.array(p.m), dtype=torch.float32, device=dev)
    h0 = torch.as_tensor(np.array(p.h), dtype=torch.float64, device=dev)
    h = torch.empty(p.n, dtype=torch.float64, device=dev)
    rho = torch.empty(p.n, dtype=torch.float32, device=dev)
    om = torch.empty(p.n, dtype=torch.float32, device=dev)
    sph.sph_density_noalloc(p.box[0], x, m, h0, h, rho, om)
    torch.cuda.synchronize()
    return {"h": h.cpu().numpy(), "rho": rho.cpu().numpy(), "omega": om.cpu().numpy()}


def test_noalloc_matches_regular_density_two_calls(torch):
    sets = [inputs.uniform(9001, seed=inputs.SEED_BASE + 31, sigma_v=0.1),
            inputs.clustered(12000, n_spheres=3, seed=inputs.SEED_BASE + 32)]
    for p in sets:  # two calls in a row share the scratch array
        ref = _regular(p)
        got = _noalloc(torch, p)
        assert np.max(np.abs(got["h"] / ref["h"] - 1)) <= TOL_H
        assert np.max(np.abs(got["rho"] / ref["rho"] - 1)) <= TOL_RHO
        assert np.max(np.abs(got["omega"] / ref["omega"] - 1)) <= TOL_OMEGA


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    p = inputs.uniform(sph.SPH_NOALLOC_MAX_PARTICLES + 1, seed=3)
    with pytest.raises(sph.SphError) as e:
        _noalloc(torch, p)
    assert e.value.code == sph.SPH_EINVAL
