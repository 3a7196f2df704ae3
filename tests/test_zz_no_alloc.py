"""The allocation-free density entry point (sph_density_noalloc) through the
C ABI, against the regular entry points (sph_init + sph_density + sph_get)
and against the FP64 oracle.

sph_density_noalloc is for callers that may not allocate device memory on
their calls (a framework that owns the GPU through its own pool, or code
where cudaMalloc/cudaFree is not allowed); it keeps its scratch in a fixed
device array shared by all calls. Two calls in a row on different particle
sets must each match, so nothing left in the scratch by the first call leaks
into the second; after a warm-up call a further call must leave the device's
free memory unchanged. This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
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


def _device_inputs(torch, p, h0=None):
    dev = torch.device("cuda")
    x = torch.as_tensor(np.array(p.x), dtype=torch.float64, device=dev)
    m = torch.as_tensor(np.array(p.m), dtype=torch.float32, device=dev)
    h0 = torch.as_tensor(np.array(p.h if h0 is None else h0), dtype=torch.float64, device=dev)
    outs = (torch.empty(p.n, dtype=torch.float64, device=dev),
            torch.empty(p.n, dtype=torch.float32, device=dev),
            torch.empty(p.n, dtype=torch.float32, device=dev))
    return x, m, h0, outs


def _noalloc(torch, p, h0=None):
    x, m, h0, (h, rho, om) = _device_inputs(torch, p, h0)
    sph.sph_density_noalloc(p.box[0], x, m, h0, h, rho, om)
    torch.cuda.synchronize()
    return {"h": h.cpu().numpy(), "rho": rho.cpu().numpy(), "omega": om.cpu().numpy()}


def _close(got, ref):
    assert np.max(np.abs(got["h"] / ref["h"] - 1)) <= TOL_H
    assert np.max(np.abs(got["rho"] / ref["rho"] - 1)) <= TOL_RHO
    assert np.max(np.abs(got["omega"] / ref["omega"] - 1)) <= TOL_OMEGA


def test_noalloc_matches_regular_density_and_oracle_two_calls(torch):
    sets = [inputs.uniform(9001, seed=inputs.SEED_BASE + 31, sigma_v=0.1),
            inputs.clustered(12000, n_spheres=3, seed=inputs.SEED_BASE + 32)]
    for p in sets:  # two calls in a row share the scratch array
        got = _noalloc(torch, p)
        _close(got, _regular(p))
        d = oracle.density(p.x, p.m.astype(np.float64), p.box[0], p.h, p.n_ngb)
        _close(got, d)


def test_noalloc_call_allocates_no_device_memory(torch):
    p = inputs.uniform(16384, seed=inputs.SEED_BASE + 33)
    x, m, h0, (h, rho, om) = _device_inputs(torch, p)
    sph.sph_density_noalloc(p.box[0], x, m, h0, h, rho, om)  # warm-up: module loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sph.sph_density_noalloc(p.box[0], x, m, h0, h, rho, om)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_inputs(torch):
    p = inputs.uniform(sph.SPH_NOALLOC_MAX_PARTICLES + 1, seed=3)
    with pytest.raises(sph.SphError) as e:
        _noalloc(torch, p)
    assert e.value.code == sph.SPH_EINVAL
    q = inputs.uniform(2000, seed=4)
    bad = np.array(q.h)
    bad[17] = 0.0
    with pytest.raises(sph.SphError) as e:
        _noalloc(torch, q, h0=bad)
    assert e.value.code == sph.SPH_EINVAL
