"""Batched solves (uneven problem sizes on concurrent streams) against single
solves and the oracle (needs a GPU).

Each problem of a batch runs the same kernels in the same order as a single
ot_ipm_solve, so its results must be identical to the single solve's up to
FP64 rounding of reductions (compared at 1e-12); one problem is also compared
with the oracle at the solver's accuracy target (cost 1e-8, rho and phi 1e-6).
A problem with mismatched masses fails alone: its status carries the error,
the others finish, and the call reports the failure.
"""
import numpy as np
import pytest
import torch

from oracle import ipm
from ot_inputs import make_density, mixture_params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SIZES = [(4, 2), (6, 3), (8, 8), (10, 5), (12, 6), (16, 4)]


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = b.detach().cpu().numpy() if isinstance(b, torch.Tensor) else np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problems():
    out = []
    for i, (n, K) in enumerate(SIZES):
        r0 = make_density(n, *mixture_params(700 + i, 1 + i % 3), 1e-4)
        r1 = make_density(n, *mixture_params(800 + i, 1 + (i + 1) % 3), 1e-4)
        out.append((n, K, r0, r1))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_equals_single_solves(gpu_lib, precision):
    from paper_2209_00315_gb300 import capi

    probs = _problems()
    meshes = {n: capi.Mesh(n) for n, _, _, _ in probs}
    opt = capi.default_options(precision=precision, final_newton_tol=1e-11, final_eps_out=1e-10)
    batch = capi.ot_ipm_solve_batched([(meshes[n], T(r0), T(r1), K) for n, K, r0, r1 in probs], options=opt,
                                      n_streams=4)
    for (n, K, r0, r1), b in zip(probs, batch):
        single = capi.ot_ipm_solve(meshes[n], T(r0), T(r1), K, options=capi.default_options(
            precision=precision, final_newton_tol=1e-11, final_eps_out=1e-10))
        assert b["status"] == 0
        assert abs(b["cost"] - single["cost"]) <= 1e-12 * abs(single["cost"])
        assert rel(b["rho"], single["rho"]) < 1e-10 and rel(b["phi"], single["phi"]) < 1e-10
        assert b["stats"]["newton_steps"] == single["stats"]["newton_steps"]
    n, K, r0, r1 = probs[3]
    d = ipm.discretise(n, K)
    ref = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(final_newton_tol=1e-11))
    b = batch[3]
    assert abs(b["cost"] - ref.cost) < 1e-8 * ref.cost
    assert rel(b["rho"], ref.rho) < 1e-6 and rel(b["phi"], ref.phi) < 1e-6


def test_batched_failure_is_isolated(gpu_lib):
    from paper_2209_00315_gb300 import capi

    probs = _problems()[:3]
    meshes = {n: capi.Mesh(n) for n, _, _, _ in probs}
    items = [(meshes[n], T(r0), T(r1), K) for n, K, r0, r1 in probs]
    bad = items[1]
    items[1] = (bad[0], bad[1], 1.5 * bad[2], bad[3])   # masses differ
    with pytest.raises(capi.OTError) as e:
        capi.ot_ipm_solve_batched(items, n_streams=2)
    assert e.value.code == 2 and "problem 1" in str(e.value)
