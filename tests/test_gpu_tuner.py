"""The multigrid autotuner (ot_tune_newton) on the GPU.

At a late-stage state of a 16x16, K = 8 mixture (the last barrier stage, where a
full solve spends most of its Newton steps) three candidate settings of
(smooth_sweeps, coarse_sweeps, lap_cycles) are timed.  Every trial reports a
positive time (or -1 if it failed), the options come back with the fastest
candidate's settings and nothing else changed, and a Newton direction computed
with the tuned options still meets the outer FGMRES tolerance: the tuner only
changes the work per step, not the answer.
"""
import numpy as np
import pytest
import torch

from ot_inputs import config_densities

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_tuner_picks_the_fastest_candidate_and_keeps_the_answer(gpu_lib):
    from paper_2209_00315_gb300 import capi

    n, K, r0, r1 = 16, 8, *config_densities("mixN", 16)[2:]
    mesh = capi.Mesh(n)
    r0d, r1d = torch.from_numpy(r0).to(DEV), torch.from_numpy(r1).to(DEV)
    base = capi.default_options(precision="mixed")
    res = capi.ot_ipm_solve(mesh, r0d, r1d, K, options=base)
    mu = res["stats"]["mu"]
    cand = [(1, 6, 1), (2, 6, 2), (3, 10, 2)]
    tuned, sec = capi.ot_tune_newton(mesh, K, mu, res["phi"], res["rho"], res["s"], r0d, r1d,
                                     options=capi.default_options(precision="mixed"), candidates=cand)
    assert len(sec) == 3 and all(t > 0 or t == -1.0 for t in sec), sec
    ok = [i for i, t in enumerate(sec) if t > 0]
    assert ok, "every candidate failed"
    best = min(ok, key=lambda i: sec[i])
    assert (tuned.smooth_sweeps, tuned.coarse_sweeps, tuned.lap_cycles) == cand[best]
    # everything else is unchanged
    for f, _ in capi.ot_options._fields_:
        if f not in ("smooth_sweeps", "coarse_sweeps", "lap_cycles"):
            assert getattr(tuned, f) == getattr(base, f), f
    # the tuned direction solves the Newton system to the outer tolerance: compare with the
    # default settings' direction at a tight tolerance
    tight = dict(final_eps_out=1e-10)
    d_ref = capi.ot_newton_solve(mesh, K, mu, res["phi"], res["rho"], res["s"], r0d, r1d,
                                 options=capi.default_options(precision="mixed", **tight))
    opt_t = capi.default_options(precision="mixed", smooth_sweeps=tuned.smooth_sweeps,
                                 coarse_sweeps=tuned.coarse_sweeps, lap_cycles=tuned.lap_cycles, **tight)
    d_tun = capi.ot_newton_solve(mesh, K, mu, res["phi"], res["rho"], res["s"], r0d, r1d, options=opt_t)
    for a, b in zip(d_tun[:3], d_ref[:3]):
        err = float(torch.linalg.norm(a - b) / max(float(torch.linalg.norm(b)), 1e-300))
        assert err < 1e-7, err
    assert d_tun[3]["fgmres_iters"] < 400
