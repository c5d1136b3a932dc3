"""The no-allocation KKT entry point (ot_kkt_apply_noalloc) against ot_kkt_apply.

Some callers cannot let a library call cudaMalloc: their device memory is
already held by another allocator (a framework's caching pool, a fixed
serving budget) or their loop cannot take the device-wide synchronisation of
cudaMalloc/cudaFree.  ot_kkt_apply_noalloc keeps its only scratch in a
file-scope device array, so the caller passes just inputs and outputs.  This
file is collected last so that a run stopping at the first failure has run
everything else already; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _state(n, K, seed):
    rng = np.random.default_rng(seed)
    N, Nc = 8 * n * n, 2 * n * n
    dev = "cuda:0"
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)  # noqa: E731
    phi = t(0.3 * rng.standard_normal((K + 1) * N))
    rho = t(rng.uniform(0.5, 2, K * Nc))
    s = t(rng.uniform(0.5, 2, K * Nc))
    r0 = t(rng.uniform(0.5, 2, Nc))
    r1 = t(rng.uniform(0.5, 2, Nc))
    x = t(rng.standard_normal((K + 1) * N + K * Nc))
    return phi, rho, s, r0, r1, x


def test_noalloc_kkt_matches_allocating_entry_point_twice(gpu_lib):
    from paper_2209_00315_gb300 import capi

    cases = [(6, 5, 1), (10, 3, 2)]  # two calls in a row with different sizes and inputs
    for n, K, seed in cases:
        phi, rho, s, r0, r1, x = _state(n, K, seed)
        mesh = capi.Mesh(n)
        ref = capi.ot_kkt_apply(mesh, K, phi, rho, s, r0, r1, x)
        out = torch.empty_like(x)
        capi.ot_kkt_apply_noalloc(n, K, phi, rho, s, r0, r1, x, out)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err < 1e-13, (n, K, err)
    # the same arguments again, after the scratch was overwritten by the other size
    phi, rho, s, r0, r1, x = _state(6, 5, 1)
    ref = capi.ot_kkt_apply(capi.Mesh(6), 5, phi, rho, s, r0, r1, x)
    out = torch.empty_like(x)
    capi.ot_kkt_apply_noalloc(6, 5, phi, rho, s, r0, r1, x, out)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref)) < 1e-13


def test_noalloc_kkt_rejects_k_beyond_its_scratch(gpu_lib):
    from paper_2209_00315_gb300 import capi

    phi, rho, s, r0, r1, x = _state(1, 1, 3)
    with pytest.raises(capi.OTError) as e:
        capi.ot_kkt_apply_noalloc(1, 4097, phi, rho, s, r0, r1, x, torch.empty_like(x))
    assert e.value.code == 1 and "4096" in str(e.value)
