"""Planted mistakes in the oracle, each of which some pin must catch.

Every case copies oracle/, ot_inputs/ and the pin tests into a temporary
directory, plants one plausible mistake in the copy (a dropped factor, a wrong
sign or time index, a transposed operand, a wrong parent cell) and runs the pins
named for it there, in a child process: at least one must fail.  The
repository's own files are never modified.  A control run of the unchanged copy
passes the same pins.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file under oracle/, text, replacement, pins (-k expression) that must catch it); a mistake that
# has to be made in several places at once to stay self-consistent lists its edits in EDITS instead.
MUTATIONS = {
    "gradient divides by |e| instead of |w|": (
        "operators.py", "sp.diags(1.0 / m.edge_dist) @ incidence(m).T", "sp.diags(1.0 / m.edge_len) @ incidence(m).T",
        "conductivity"),
    "projector P exchanged for its transpose": (
        "operators.py", "np.outer(mc, np.ones(self.Nc))", "np.outer(np.ones(self.Nc), mc)", "graded"),
    "C = M' diag(rho/s) instead of diag(s/rho)": (
        "operators.py", "mc * np.asarray(s) / np.asarray(rho)", "mc * np.asarray(rho) / np.asarray(s)",
        "projected_system"),
    "B takes grad phi of the wrong slice": (
        "operators.py", "blocks[k][k] = -JtM / dt + 0.5 * Gk\n", "blocks[k][k] = -JtM / dt + 0.5 * Gk1\n",
        "jacobian_matches"),
    "time average in rho~ off-centre": (
        "operators.py", "avg = 0.5 * (r[1:] + r[:-1])", "avg = 0.7 * r[1:] + 0.3 * r[:-1]", "symmetries"),
    "end densities exchanged in the space-time density array": (
        "operators.py", "return np.vstack([rho0[None, :], self.rho_slices(rho), rho1[None, :]])",
        "return np.vstack([rho1[None, :], self.rho_slices(rho), rho0[None, :]])", "duality_gap"),
    "rho~ from the later slice alone instead of the time average": (
        "operators.py", "avg = 0.5 * (r[1:] + r[:-1])", "avg = r[1:]", "jacobian_matches"),
    "B~ spatial term with the wrong sign": (
        "operators.py", "blocks[j][j - 1] = -MJ / dt + 0.5 * S", "blocks[j][j - 1] = -MJ / dt - 0.5 * S", "btilde"),
    "B~ time term with the wrong sign on the current slice": (
        "operators.py", "blocks[j][j] = MJ / dt + 0.5 * S", "blocks[j][j] = -MJ / dt + 0.5 * S", "btilde"),
    "A~^k from the time average of rho^k and rho^(k+1) instead of rho^k": (
        "operators.py", "return sp.block_diag([weighted_laplacian(c, Rc @ R[k]) for k in range(self.K)]).tocsr()",
        "return sp.block_diag([weighted_laplacian(c, Rc @ (0.5 * (R[k] + R[min(k + 1, self.K - 1)])))"
        " for k in range(self.K)]).tocsr()", "depends_on_rho_k"),
    "B~ spatial term with grad phi of the previous slice": (
        "operators.py", "S = (Rf.T @ sp.diags(self.W * (self.grad @ P[j])) @ self.grad @ self.J).tocsr()",
        "S = (Rf.T @ sp.diags(self.W * (self.grad @ P[max(j - 1, 0)])) @ self.grad @ self.J).tocsr()", "btilde"),
    "BB: y without M'^-1": (
        "operators.py", "y = (d.A_tilde_block(rho) @ z) / np.tile(d.t.coarse.area, d.K)",
        "y = d.A_tilde_block(rho) @ z", "exact_bb"),
    "BB Schur approximation with the wrong sign": (
        "operators.py", "- sp.diags(np.asarray(rho)) @ B @ Minv", "+ sp.diags(np.asarray(rho)) @ B @ Minv",
        "exact_bb"),
    "SIMPLE: Schur complement with the wrong sign of the C term": (
        "operators.py", "S = -(P @ d.C_block(rho, s) @ P.T + Bp", "S = -(-P @ d.C_block(rho, s) @ P.T + Bp",
        "simple_application"),
    "SIMPLE: back substitution without A^-1": (
        "operators.py", "return x1 - (Bp.T @ y) / Ad, y", "return x1 - Bp.T @ y, y", "simple_application"),
    "degenerate |w| doubled": (
        "mesh.py", "edge_dist = np.where(degenerate, bdist, dist)", "edge_dist = np.where(degenerate, 2 * bdist, dist)",
        "geometry"),
    "edge weight lambda measured from the right cell's point (1/2 on the right-triangle grid)": (
        "mesh.py", "d_left = _point_line_distance(centre[left], va, vb)",
        "d_left = _point_line_distance(centre[right], va, vb)", "circumcentric"),
    "circumcentre y with a sign error": (
        "mesh.py", "uy = (a2 * (c[:, 0] - b[:, 0])", "uy = (a2 * (b[:, 0] - c[:, 0])", "geometry"),
    "two children per cell given to the next parent": (
        "mesh.py", "            parent.append(c)\n", "            parent.append(c if t[0] != ab else (c + 1) % len(tri))\n",
        "nesting"),
    "continuity equation with the wrong sign of the time difference": (
        "ipm.py", "Fphi[k] = -(d.M @ (d.J @ (R[k + 1] - R[k]))) / dt", "Fphi[k] = +(d.M @ (d.J @ (R[k + 1] - R[k]))) / dt",
        "jacobian_matches"),
    "Hamilton-Jacobi time difference reversed": (
        "ipm.py", "JtM @ (P[k + 1] - P[k]) / dt", "JtM @ (P[k] - P[k + 1]) / dt", "jacobian_matches"),
    "complementarity row of the Jacobian with diag(s) and diag(rho) exchanged": (
        "ipm.py", "[Z(Nr, Np), sp.diags(np.asarray(s)), sp.diags(np.asarray(rho))],",
        "[Z(Nr, Np), sp.diags(np.asarray(rho)), sp.diags(np.asarray(s))],", "jacobian_matches"),
    "complementarity rho s = 2 mu": (
        "ipm.py", "Fs = R[1:-1] * S - mu", "Fs = R[1:-1] * S - 2 * mu", "uniform"),
    "stopping rule compares mu with the tolerance, without the gap's factor |Omega| K/(K+1)": (
        "ipm.py", "while mu * area_total * K / (K + 1) > opt.gap_tol", "while mu * area_total > opt.gap_tol",
        "stops_at_the_first_stage"),
    "fraction to the boundary over rho alone, not over s": (
        "ipm.py", "alpha = min(step_length(rho, drho, opt.tau), step_length(s, ds, opt.tau))",
        "alpha = step_length(rho, drho, opt.tau)", "barycentre"),
    "cost scaled by 1/K instead of dt": (
        "ipm.py", "return d.dt * total", "return total / d.K", "duality_gap"),
    "dual value with the end densities exchanged": (
        "ipm.py", "term = float(P[-1] @ (MJ @ rho1)) - float(P[0] @ (MJ @ rho0))",
        "term = float(P[-1] @ (MJ @ rho0)) - float(P[0] @ (MJ @ rho1))", "duality_gap"),
    "Hamilton-Jacobi kinetic term doubled": (
        "ipm.py", "+ 0.25 * (d.RT @ (g0 ** 2 + g1 ** 2))", "+ 0.5 * (d.RT @ (g0 ** 2 + g1 ** 2))",
        "jacobian_matches"),
    "slack enters F_rho without the coarse mass matrix": (
        "ipm.py", "+ d.Mc @ S[k]", "+ S[k]", "jacobian_matches"),
    "slack weighted by 1/N' instead of the cell areas (equal on the uniform grid)": (
        "ipm.py", "+ d.Mc @ S[k]", "+ S[k] / d.Nc", "exact_solution_on_a_graded_mesh"),
    "R_T weighted by |e|/|w| instead of |e||w|": (
        "operators.py", "sp.diags(f.edge_dist * f.edge_len)", "sp.diags(f.edge_len / f.edge_dist)",
        "symmetric_saddle"),
    "dual value's boundary kinetic terms weighted dt/2 instead of dt/4": (
        "ipm.py", "return term - 0.25 * d.dt * corr", "return term - 0.5 * d.dt * corr", "identity_at_any_point"),
    "cost without the 1/2 of the kinetic energy": (
        "ipm.py", "total += 0.5 * float(np.dot(d.W * rt[k], g * g))", "total += float(np.dot(d.W * rt[k], g * g))",
        "identity_at_any_point"),
    "adjoint: initial-time flux with the wrong sign": (
        "adjoint.py", "(MJ / d.dt + flux(0))", "(MJ / d.dt - flux(0))", "adjoint_gradient_matches"),
    "adjoint: final-time flux with the wrong sign": (
        "adjoint.py", "(-MJ / d.dt + flux(d.K))", "(-MJ / d.dt - flux(d.K))", "adjoint_gradient_matches"),
    "adjoint: kinetic partial doubled": (
        "adjoint.py", "e = [0.25 * d.dt *", "e = [0.5 * d.dt *", "adjoint_gradient_matches"),
}

# ([(file, text, replacement), ...], pins): the same mistake made consistently in the residual and in
# the Jacobian, so that the Jacobian-versus-differences pin cannot see it
EDITS = {
    "time term of F_rho as M'J^T (the printed order) in F_rho and in B": (
        [("ipm.py", "JtM = d.J.T @ d.M", "JtM = d.Mc @ d.J.T"),
         ("operators.py", "JtM = (self.J.T @ self.M).tocsr()", "JtM = (self.Mc @ self.J.T).tocsr()")],
        "symmetric_saddle"),
    "slack weighted by 1/N' in F_rho, in the Jacobian and in C": (
        [("ipm.py", "+ d.Mc @ S[k]", "+ S[k] / d.Nc"),
         ("operators.py", "return sp.diags(np.tile(self.t.coarse.area, self.K))",
          "return sp.diags(np.full(self.K * self.Nc, 1.0 / self.Nc))"),
         ("operators.py", "mc = np.tile(self.t.coarse.area, self.K)\n        return sp.diags(mc * np.asarray(s)",
          "mc = np.full(self.K * self.Nc, 1.0 / self.Nc)\n        return sp.diags(mc * np.asarray(s)")],
        "exact_solution_on_a_graded_mesh"),
}


def _copy(dst):
    for d in ("oracle", "ot_inputs"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("__pycache__", "*.so", "_build"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _run_pins(repo, expr):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    env.pop("PYTHONPATH", None)
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                           "-p", "no:cacheprovider", "-k", expr], cwd=repo, env=env, capture_output=True,
                          text=True, timeout=600)


def test_unmutated_copy_passes_the_pins_used_below(tmp_path):
    _copy(str(tmp_path))
    expr = " or ".join(sorted({m[3] for m in MUTATIONS.values()} | {m[1] for m in EDITS.values()}))
    r = _run_pins(str(tmp_path), expr)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


def _plant(repo, edits):
    for f, old, new in edits:
        path = os.path.join(repo, "oracle", f)
        src = open(path).read()
        assert src.count(old) == 1, "the text to mutate must occur exactly once"
        open(path, "w").write(src.replace(old, new, 1))


@pytest.mark.parametrize("name", list(MUTATIONS) + list(EDITS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    if name in MUTATIONS:
        f, old, new, expr = MUTATIONS[name]
        edits = [(f, old, new)]
    else:
        edits, expr = EDITS[name]
    _copy(str(tmp_path))
    _plant(str(tmp_path), edits)
    r = _run_pins(str(tmp_path), expr)
    assert r.returncode == 1 and " failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
