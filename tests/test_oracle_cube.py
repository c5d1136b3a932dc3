"""The oracle's 3D Cartesian variant (test 4 of Sec. 4.1: cubes, J = I), pinned on the CPU.

The same operators as in 2D, built from a cube grid whose TPFA fields (cell
measure, face measure, centre distance, weight 1/2) replace the triangle
geometry; density and potential live on the same grid, so the injection J is
the identity.  The pins: the grid's geometry in closed form, the Jacobian
against central differences and its symmetric saddle form, the uniform-density
exact solution, the duality identity at any point, and on the paper's 3D
Gaussians (sigma 0.1 at (0.3,0.3,0.3) -> (0.7,0.7,0.7), floor 1e-3) mass,
positivity, the barrier gap, barycentres on a straight line at constant speed,
the symmetries of the problem, and the cost decreasing towards |m1 - m0|^2/2.
"""
import numpy as np
import pytest

from oracle import ipm
from ot_inputs import cube_config_densities, make_cube_density


def _random_state(d, seed=0):
    rng = np.random.default_rng(seed)
    phi = 0.3 * rng.standard_normal((d.K + 1) * d.N)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    rho = ipm.renormalise(d, rng.uniform(0.5, 2, d.K * d.Nc), r0)
    s = rng.uniform(0.5, 2, d.K * d.Nc)
    return phi, rho, s, r0, r1


@pytest.mark.parametrize("n", [1, 2, 3])
def test_cube_grid_geometry(n):
    """n^3 cells of volume h^3, 3 n^2 (n-1) interior faces of area h^2 at centre
    distance h, and for every cell sum_faces |e| d_{K,e} n_e n_e^T = |K| I over its
    interior faces plus the boundary ones (d = h/2), i.e. the interior faces alone
    give |K| I minus h^3/2 per boundary face direction."""
    d = ipm.discretise_cube(n, 1)
    m = d.t.fine
    h = 1.0 / n
    assert m.ncell == n ** 3 and m.nedge == 3 * n * n * (n - 1)
    assert np.allclose(m.area, h ** 3) and abs(m.area.sum() - 1.0) < 1e-14
    assert np.allclose(m.edge_len, h * h) and np.allclose(m.edge_dist, h) and np.allclose(m.edge_lambda, 0.5)
    T = np.zeros((m.ncell, 3, 3))
    for (a, b), ax in zip(m.edge_cells, m.edge_axis):
        assert np.isclose(abs(m.centre[b] - m.centre[a]).sum(), h)
        nn = np.zeros(3)
        nn[ax] = 1.0
        for c in (a, b):
            T[c] += h * h * (h / 2) * np.outer(nn, nn)
    ijk = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)[..., ::-1].reshape(-1, 3)
    for c in range(m.ncell):
        boundary = [int(ijk[c, a] == 0) + int(ijk[c, a] == n - 1) for a in range(3)]
        expect = np.diag([h ** 3 - bnd * h ** 3 / 2 for bnd in boundary])
        assert np.allclose(T[c], expect, atol=1e-15)
    assert (d.J - np.eye(m.ncell)).__abs__().max() == 0


def test_cube_jacobian_matches_central_differences_and_is_a_symmetric_saddle():
    d = ipm.discretise_cube(2, 2)
    phi, rho, s, r0, r1 = _random_state(d)
    Np, Nr = (d.K + 1) * d.N, d.K * d.Nc
    Jm = ipm.jacobian(d, phi, rho, s, r0, r1).toarray()
    x = np.concatenate([phi, rho, s])
    F = lambda x: np.concatenate(ipm.residual(d, x[:Np], x[Np:Np + Nr], x[Np + Nr:], r0, r1, 0.3))  # noqa
    h = 1e-6
    FD = np.empty_like(Jm)
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        FD[:, i] = (F(x + e) - F(x - e)) / (2 * h)
    assert np.abs(FD - Jm).max() < 1e-7 * np.abs(Jm).max()
    assert np.allclose(ipm.dFphi_drho(d, phi).toarray(), d.B_block(phi).T.toarray(), atol=1e-13)


def test_cube_uniform_densities_exact_solution():
    """rho_in = rho_f = c: rho^k = c, s = mu/c, phi^k = -(k-1) dt mu/c + const, C = 0."""
    n, K, c = 3, 3, 1.0
    d = ipm.discretise_cube(n, K)
    r0 = np.full(d.Nc, c)
    res = ipm.ipm_solve(d, r0, r0.copy(), ipm.IPMOptions(final_newton_tol=1e-12))
    assert all(steps == 1 for _, steps, _ in res.stages)
    assert np.allclose(res.rho, c, rtol=0, atol=1e-13)
    assert np.allclose(res.s, res.mu / c, rtol=1e-12)
    k = np.arange(K + 1)
    assert np.allclose(res.phi, ipm.phi_gauge(d, np.repeat(-k * d.dt * res.mu / c, d.N)), atol=1e-14)
    assert abs(res.cost) < 1e-25
    assert np.isclose(res.cost - res.dual, res.mu * K / (K + 1), rtol=1e-12)


def test_cube_duality_gap_identity_at_any_point():
    """C - D - mu |Omega| K/(K+1) = dt [sum phi.F_phi - sum rho.F_rho + sum |c'|.F_s] off the solution."""
    n, K = 3, 3
    d = ipm.discretise_cube(n, K)
    phi, rho, s, r0, r1 = _random_state(d, seed=5)
    mu = 0.29
    Fphi, Frho, Fs = ipm.residual(d, phi, rho, s, r0, r1, mu)
    C = ipm.cost(d, phi, rho, r0, r1)
    D = ipm.dual_value(d, phi, r0, r1)
    area = d.t.coarse.area
    rhs = d.dt * (phi @ Fphi - rho @ Frho + np.tile(area, K) @ Fs)
    lhs = C - D - mu * area.sum() * K / (K + 1)
    scale = abs(C) + abs(D) + d.dt * (abs(phi) @ abs(Fphi) + abs(rho) @ abs(Frho))
    assert abs(lhs - rhs) < 1e-13 * scale


@pytest.fixture(scope="module")
def gauss_cubes():
    out = {}
    for n in (4, 6):
        _, K, r0, r1 = cube_config_densities("gauss_cubeN", n)
        d = ipm.discretise_cube(n, K)
        out[n] = (d, r0, r1, ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(final_newton_tol=1e-11)))
    return out


def test_cube_gaussians_converge_with_mass_positivity_and_gap(gauss_cubes):
    for n, (d, r0, r1, res) in gauss_cubes.items():
        R = res.rho.reshape(d.K, d.Nc)
        assert np.allclose(R @ d.t.coarse.area, d.t.coarse.area @ r0, rtol=0, atol=1e-14)
        assert res.rho.min() > 0 and res.s.min() > 0
        gap = res.mu * d.area_total * d.K / (d.K + 1)
        assert abs((res.cost - res.dual) - gap) < 1e-8 * gap + 1e-12 * res.cost   # C - D cancels 13 digits
        assert ipm.residual_norm(ipm.residual(d, res.phi, res.rho, res.s, r0, r1, res.mu)) < 1e-10


def test_cube_gaussian_cost_decreases_towards_the_translation_cost(gauss_cubes):
    """Equal Gaussians translated by m1 - m0 = (0.4, 0.4, 0.4): C -> |m1 - m0|^2 / 2 = 0.24
    on R^3 without a floor; on the unit cube with the 1e-3 floor the discrete costs come
    down towards it as the grid is refined (0.2838 at 4^3, K = 3; 0.2704 at 6^3, K = 5;
    0.2544 at 8^3, K = 7, the last too slow for this suite)."""
    c4, c6 = gauss_cubes[4][3].cost, gauss_cubes[6][3].cost
    assert 0.24 < c6 < c4 < 0.3
    assert (c6 - 0.24) < 0.8 * (c4 - 0.24)


def test_cube_gaussian_barycentres_move_on_a_straight_line(gauss_cubes):
    """Momentum is conserved along a W2 geodesic: the barycentre of rho^k lies on the
    segment from b_in to b_f at t_k = k/(K+1), to 1% of the displacement at 6^3."""
    d, r0, r1, res = gauss_cubes[6]
    a, c = d.t.coarse.area, d.t.coarse.centre
    b0, b1 = (r0 * a) @ c / (r0 @ a), (r1 * a) @ c / (r1 @ a)
    R = res.rho.reshape(d.K, d.Nc)
    t = np.arange(1, d.K + 1) / (d.K + 1)
    B = (R * a) @ c / (R @ a)[:, None]
    dev = np.abs(B - ((1 - t)[:, None] * b0 + t[:, None] * b1)).max()
    assert dev < 0.01 * np.abs(b1 - b0).max()


def test_cube_solution_respects_time_reversal_and_axis_permutations():
    """Swapping rho_in and rho_f reverses rho in time and maps phi^k to -phi^(K+2-k);
    exchanging two coordinate axes permutes the cells and leaves the solution of
    the (axis-symmetric) diagonal Gaussian test in place; both to 1e-9."""
    n = 4
    _, K, g0, g1 = cube_config_densities("gauss_cubeN", n)
    d = ipm.discretise_cube(n, K)
    # asymmetric data for the time reversal
    r0 = make_cube_density(n, [(0.3, 0.4, 0.5)], [0.15], [1.0], 1e-3)
    r1 = make_cube_density(n, [(0.6, 0.7, 0.45)], [0.12], [1.0], 1e-3)
    opt = ipm.IPMOptions(final_newton_tol=1e-12)
    fwd = ipm.ipm_solve(d, r0, r1, opt)
    bwd = ipm.ipm_solve(d, r1, r0, opt)
    R, Rb = fwd.rho.reshape(K, -1), bwd.rho.reshape(K, -1)
    assert np.abs(R - Rb[::-1]).max() < 1e-9 * np.abs(R).max()
    P, Pb = d.phi_slices(fwd.phi), d.phi_slices(bwd.phi)
    assert np.abs(P + Pb[::-1]).max() < 1e-9 * np.abs(P).max()
    # axis exchanges on the symmetric test: cell (i, j, k) -> (j, i, k) and (k, j, i)
    res = ipm.ipm_solve(d, g0, g1, opt)
    idx = np.arange(n ** 3).reshape(n, n, n)          # [k][j][i]
    for perm in (idx.transpose(0, 2, 1).ravel(), idx.transpose(2, 1, 0).ravel()):
        Rs = res.rho.reshape(K, -1)
        assert np.abs(Rs - Rs[:, perm]).max() < 1e-9 * np.abs(Rs).max()


@pytest.mark.slow
def test_cube_preconditioner_iteration_trends_along_the_barrier_path():
    """Sec. 4.2-4.3 on the 3D variant, with exact inner solves: at the first Newton
    step of each mu stage (4^3 cubes, K = 3, the 3D Gaussians) the BB-preconditioned
    GMRES needs more iterations as mu decreases (measured 4 -> 13), and SIMPLE fewer
    over the late stages, ending below BB (measured 15 at its peak -> 9)."""
    from oracle import operators as ops
    from test_oracle_pins import _gmres_right

    n = 4
    _, K, r0, r1 = cube_config_densities("gauss_cubeN", n)
    d = ipm.discretise_cube(n, K)
    opt = ipm.IPMOptions()
    phi, rho, s = ipm.initial_point(d, r0, r1, opt.mu0)
    mu = opt.mu0
    bb, simple = [], []
    for _ in range(ipm.stage_count(K, opt, d.area_total)):
        F = ipm.residual(d, phi, rho, s, r0, r1, mu)
        f0 = fn = ipm.residual_norm(F)
        first = True
        while fn > opt.newton_tol * max(1.0, f0):
            if first:
                Kp = d.projected_kkt(phi, rho, s, r0, r1)
                gt = -F[1] + np.tile(d.t.coarse.area, K) * F[2] / rho
                b = np.concatenate([-F[0], d.P_block() @ gt])
                st = (phi, rho, s, r0, r1)
                bb.append(_gmres_right(lambda x: Kp @ x, b, lambda v: np.concatenate(ops.bb_apply_exact(d, *st, v))))
                simple.append(_gmres_right(lambda x: Kp @ x, b,
                                           lambda v: np.concatenate(ops.simple_apply_exact(d, *st, v))))
                first = False
            dphi, drho, ds, _ = ipm.newton_direction(d, phi, rho, s, r0, r1, mu)
            a = min(ipm.step_length(rho, drho, opt.tau), ipm.step_length(s, ds, opt.tau))
            phi, rho, s = phi + a * dphi, ipm.renormalise(d, rho + a * drho, r0), s + a * ds
            F = ipm.residual(d, phi, rho, s, r0, r1, mu)
            fn = ipm.residual_norm(F)
        mu *= opt.mu_factor
    assert len(bb) == 10
    assert all(b1 <= b2 for b1, b2 in zip(bb, bb[1:])) and bb[-1] >= 3 * bb[0]
    peak = int(np.argmax(simple))
    assert all(a >= b for a, b in zip(simple[peak:], simple[peak + 1:]))
    assert simple[-1] < bb[-1]
