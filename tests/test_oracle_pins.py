"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
identity derived independently of the code, a brute-force derivative, a
special case with a known solution, or a value printed in the paper.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import ipm, mesh, operators as ops
from ot_inputs import make_density, mixture_params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- geometry
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_mesh_counts_and_nesting(n):
    """N' = 2n^2, N = 4N' = 8n^2, N'_e = 3n^2-2n, N_e = 12n^2-4n = 2N'_e + 4N' - ... (Sec. 2.1)."""
    t = mesh.two_level_square(n)
    assert t.coarse.ncell == 2 * n * n and t.fine.ncell == 8 * n * n
    assert t.coarse.nedge == 3 * n * n - 2 * n
    # fine interior edges: each coarse interior edge splits in two, plus 3 new edges per coarse cell
    assert t.fine.nedge == 2 * t.coarse.nedge + 3 * t.coarse.ncell
    assert np.isclose(t.coarse.area.sum(), 1.0) and np.isclose(t.fine.area.sum(), 1.0)
    counts = np.bincount(t.parent, minlength=t.coarse.ncell)
    assert np.all(counts == 4)
    child_area = np.bincount(t.parent, weights=t.fine.area)
    assert np.allclose(child_area, t.coarse.area, rtol=0, atol=1e-15)
    # J: every fine cell lies inside its parent (positive barycentric coordinates of its centroid)
    a, b, c = (t.coarse.xy[t.coarse.tri[t.parent, i]] for i in range(3))
    g = t.fine.bary
    cross = lambda u, v: u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]  # noqa: E731
    lam = np.stack([cross(b - g, c - g), cross(c - g, a - g), cross(a - g, b - g)], 1)
    assert np.all(lam > 0.05 * np.abs(lam).sum(1, keepdims=True))


@pytest.mark.parametrize("n", [2, 4])
def test_geometry_closed_form(n):
    """Right triangles: circumcentre = hypotenuse midpoint, |e|/|w| = 1 on legs, 3 on hypotenuses
    (barycentre distance sqrt(2) h/3, reading R1), lambda = 1/2 everywhere (reading R2)."""
    for m, tm in ((n, mesh.build_mesh(*mesh.square_grid(n))), (2 * n, mesh.two_level_square(n).fine)):
        h = 1.0 / m
        p = tm.xy[tm.tri]
        side = np.stack([np.hypot(*(p[:, (k + 1) % 3] - p[:, k]).T) for k in range(3)], 1)
        hyp = np.argmax(side, 1)
        mid = np.array([(p[c, hyp[c]] + p[c, (hyp[c] + 1) % 3]) / 2 for c in range(tm.ncell)])
        assert np.allclose(tm.centre, mid, atol=1e-14)
        legs = np.isclose(tm.edge_len, h)
        diag = np.isclose(tm.edge_len, np.sqrt(2) * h)
        assert np.all(legs | diag)
        assert np.array_equal(diag, tm.degenerate)
        assert np.allclose(tm.edge_dist[legs], h)
        assert np.allclose(tm.edge_dist[diag], np.sqrt(2) * h / 3)
        assert np.allclose(tm.edge_lambda, 0.5)


def test_edge_weights_satisfy_the_circumcentric_identity_on_an_acute_mesh():
    """Reading R2 on a generic mesh.  For a triangle K with its circumcentre, the
    distances d_{K,e} to its three edges satisfy sum_e |e| d_{K,e} n_e n_e^T = |K| I
    (the circumcentric form of the divergence theorem).  With lambda_e = d_{K,e}/|w_e|
    on the left cell and 1 - lambda_e on the right, every acute triangle whose three
    edges are interior must reproduce |K| I.  On the right-triangle grid lambda is
    1/2 everywhere, so only an irregular mesh can tell the two cells apart: a
    jittered triangular lattice, Delaunay-triangulated."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(3)
    h = 0.125
    lattice = np.array([((i + 0.5 * (j % 2)) * h, j * h * np.sqrt(3) / 2) for j in range(10) for i in range(10)])
    xy = lattice + rng.uniform(-0.12, 0.12, lattice.shape) * h
    tri = Delaunay(xy).simplices.copy()
    p = xy[tri]
    e1, e2 = p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]
    cw = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0] < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    p = xy[tri]
    # acute: at every vertex the two edges leaving it have a positive dot product
    acute = np.min([np.einsum("ij,ij->i", p[:, (k + 1) % 3] - p[:, k], p[:, (k + 2) % 3] - p[:, k])
                    for k in range(3)], 0) > 1e-3 * h * h
    m = mesh.build_mesh(xy, tri)
    assert not m.degenerate.any()
    T = np.zeros((m.ncell, 2, 2))
    count = np.zeros(m.ncell, dtype=int)
    for e, (L, R) in enumerate(m.edge_cells):
        a, b = sorted(set(tri[L].tolist()) & set(tri[R].tolist()))  # the edge's two vertices
        t = xy[b] - xy[a]
        nn = np.outer([t[1], -t[0]], [t[1], -t[0]]) / float(t @ t)  # unit normal from the vertices
        T[L] += m.edge_len[e] * m.edge_lambda[e] * m.edge_dist[e] * nn
        T[R] += m.edge_len[e] * (1.0 - m.edge_lambda[e]) * m.edge_dist[e] * nn
        count[L] += 1
        count[R] += 1
    sel = (count == 3) & acute
    assert sel.sum() > 100
    assert np.abs(T[sel] - m.area[sel, None, None] * np.eye(2)).max() < 1e-12 * m.area[sel].max()
    # the weights are not all 1/2 here, so the test can see which cell is which
    assert np.ptp(m.edge_lambda[sel[m.edge_cells[:, 0]] & sel[m.edge_cells[:, 1]]]) > 0.1


def test_effective_conductivity_closed_form():
    """Homogenised x-conductivity of the unit-coefficient TPFA Laplacian on this mesh.

    With transmissibility T_d = 3 on diagonals and 1 on legs, the periodic cell
    problem gives K = diag(1, T_d/(T_d+2)) in the (1,1),(1,-1) frame, so a
    walled strip conducts K_xx - K_xy^2/K_yy = T_d/(T_d+1) = 3/4 along x.
    A wrong |w| on either edge type moves this limit.
    """
    got = []
    for m in (8, 16):
        tm = mesh.build_mesh(*mesh.square_grid(m))
        A = ops.weighted_laplacian(tm, np.ones(tm.nedge)).tolil()
        c = tm.bary
        b = np.zeros(tm.ncell)
        left, right = c[:, 0] < 1.0 / m, c[:, 0] > 1 - 1.0 / m
        b[left] = tm.area[left] / tm.area[left].sum()
        b[right] = -tm.area[right] / tm.area[right].sum()
        A[0, :] = 0
        A[0, 0] = 1
        b[0] = 0
        u = spla.spsolve(A.tocsr(), b)
        mid = (c[:, 0] > 0.25) & (c[:, 0] < 0.75)
        got.append(-1.0 / np.polyfit(c[mid, 0], u[mid], 1)[0])
    assert abs(got[1] - 0.75) < abs(got[0] - 0.75) < 0.02
    assert abs(got[1] - 0.75) < 0.005


def test_operator_identities():
    """div = -grad^T diag(|w||e|), A 1 = 0, J^T M J = M', J^T M 1 = |c'|, P^2 = P, P M'E'^T = 0."""
    d = ipm.discretise(3, 3)
    f = d.t.fine
    D1 = d.div.toarray()
    D2 = -(d.grad.T @ sp.diags(f.edge_dist * f.edge_len)).toarray()
    assert np.allclose(D1, D2, atol=1e-14)
    rng = np.random.default_rng(1)
    A = ops.weighted_laplacian(f, rng.uniform(0.1, 2, f.nedge))
    assert np.allclose(A @ np.ones(d.N), 0, atol=1e-13)
    assert np.allclose((A - A.T).toarray(), 0, atol=1e-14)
    assert np.allclose((d.J.T @ d.M @ d.J).toarray(), d.Mc.toarray(), atol=1e-16)
    assert np.allclose(d.J.T @ (d.M @ np.ones(d.N)), d.t.coarse.area)
    P = d.P_block().toarray()
    assert np.allclose(P @ P, P, atol=1e-14)
    mcE = np.kron(np.eye(d.K), d.t.coarse.area[:, None])
    assert np.allclose(P @ mcE, 0, atol=1e-14)
    # P^T maps into mass-free vectors: |c'|^T (P^T y)^k = 0
    y = rng.standard_normal(d.K * d.Nc)
    z = (P.T @ y).reshape(d.K, d.Nc)
    assert np.allclose(z @ d.t.coarse.area, 0, atol=1e-15)
    # R_E is a weighted mean: it preserves constants
    assert np.allclose(d.RE @ np.ones(d.Nc), 1.0)


def _graded_discretisation(n, K):
    """The n x n diagonal grid of the unit square with x moved to x + 0.15 x (1 - x):
    the domain and its area stay the same, the coarse cells' areas differ."""
    xy, tri = mesh.square_grid(n)
    xy = xy.copy()
    xy[:, 0] += 0.15 * xy[:, 0] * (1.0 - xy[:, 0])
    fxy, ftri, parent = mesh.refine4(xy, tri)
    t = mesh.TwoLevelMesh(mesh.build_mesh(xy, tri), mesh.build_mesh(fxy, ftri), parent, n)
    return ops.Discretisation(t, K)


def test_operator_identities_on_a_graded_mesh():
    """The same identities where the coarse cells differ in area (the grid stretched
    along x), which tells P = I - M' E'^T E'/|Omega| from its transpose: P kills
    the per-slice mass vectors M'E'^T, P^T y has zero mass in every slice, P^2 = P,
    and J^T M J = M' for any midpoint 4-split."""
    d = _graded_discretisation(3, 2)
    area = d.t.coarse.area
    assert area.max() - area.min() > 0.01
    P = d.P_block().toarray()
    mcE = np.kron(np.eye(d.K), area[:, None])
    assert np.abs(P @ mcE).max() < 1e-15 and np.abs(P @ P - P).max() < 1e-14
    y = np.random.default_rng(4).standard_normal(d.K * d.Nc)
    assert np.abs((P.T @ y).reshape(d.K, d.Nc) @ area).max() < 1e-15
    assert np.allclose((d.J.T @ d.M @ d.J).toarray(), d.Mc.toarray(), atol=1e-16)
    assert abs(d.area_total - 1.0) < 1e-14


# ----------------------------------------------------------------- Jacobian
def _random_state(d, seed=0):
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((d.K + 1) * d.N)
    rho = rng.uniform(0.5, 2, d.K * d.Nc)
    s = rng.uniform(0.5, 2, d.K * d.Nc)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    return phi, rho, s, r0, r1


def test_jacobian_matches_central_differences():
    d = ipm.discretise(2, 2)
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


def test_jacobian_is_symmetric_saddle():
    """dF_phi/drho equals B^T = (dF_rho/dphi)^T: the Jacobian is a symmetric saddle (Sec. 3)."""
    d = ipm.discretise(3, 3)
    phi, rho, s, r0, r1 = _random_state(d, 3)
    B = d.B_block(phi)
    assert np.allclose(ipm.dFphi_drho(d, phi).toarray(), B.T.toarray(), atol=1e-13)


def test_kernel_of_jacobian_is_global_constant():
    """Remark (kernel): the Jacobian kernel is spanned by (1, 0, 0)."""
    d = ipm.discretise(1, 2)
    phi, rho, s, r0, r1 = _random_state(d, 5)
    Jm = ipm.jacobian(d, phi, rho, s, r0, r1).toarray()
    sv = np.linalg.svd(Jm, compute_uv=False)
    assert sv[-1] < 1e-12 * sv[0] and sv[-2] > 1e-6 * sv[0]
    Np = (d.K + 1) * d.N
    e = np.zeros(Jm.shape[0])
    e[:Np] = 1
    assert np.abs(Jm @ e).max() < 1e-12


def _disc(geom, n, K):
    """The 2D two-level triangle discretisation or the 3D cube grid of test 4."""
    return ipm.discretise(n, K) if geom == "tri" else ipm.discretise_cube(n, K)


# ------------------------------------------------------- projected system
@pytest.mark.parametrize("geom,n,K", [("tri", 1, 1), ("tri", 2, 2), ("tri", 2, 3), ("cube", 2, 2)])
def test_projected_system_reproduces_newton_direction(geom, n, K):
    """The projected system (Sec. 4.3.1) plus the per-slice constants of the
    splitting (reading R10) reproduces the exact Newton direction (dense LU),
    on triangles and on the cube grid of the 3D variant."""
    d = _disc(geom, n, K)
    rng = np.random.default_rng(7 + n + K)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    phi = 0.3 * rng.standard_normal((d.K + 1) * d.N)
    rho = rng.uniform(0.5, 2, d.K * d.Nc)
    rho = ipm.renormalise(d, rho, r0)
    s = rng.uniform(0.5, 2, d.K * d.Nc)
    mu = 0.1
    dphi, drho, ds, dropped = ipm.newton_direction(d, phi, rho, s, r0, r1, mu)
    assert abs(dropped) < 1e-12
    # dense LU of the full (singular, bordered) Jacobian as an independent route
    Jm = ipm.jacobian(d, phi, rho, s, r0, r1).toarray()
    F = np.concatenate(ipm.residual(d, phi, rho, s, r0, r1, mu))
    Np, Nr = (d.K + 1) * d.N, d.K * d.Nc
    w = np.zeros(len(F))
    w[:Np] = np.tile(d.t.fine.area, d.K + 1)
    e = np.zeros(len(F))
    e[:Np] = 1
    big = np.block([[Jm, e[:, None]], [w[None, :], np.zeros((1, 1))]])
    sol = np.linalg.solve(big, np.concatenate([-F, [0]]))
    assert np.allclose(sol[:Np], dphi, atol=1e-10)
    assert np.allclose(sol[Np:Np + Nr], drho, atol=1e-10)
    assert np.allclose(sol[Np + Nr:-1], ds, atol=1e-10)
    # projected system
    f, g, h = -F[:Np], -F[Np:Np + Nr], -F[Np + Nr:]
    gt = g - np.tile(d.t.coarse.area, d.K) * h / rho
    Kp = d.projected_kkt(phi, rho, s, r0, r1).toarray()
    P = d.P_block().toarray()
    rhs = np.concatenate([f, P @ gt])
    x = np.linalg.lstsq(Kp, rhs, rcond=None)[0]
    dphi_hat, drho_p = x[:Np], P.T @ x[Np:]
    assert np.allclose(drho_p, drho, atol=1e-10)
    # reading R10: add per-slice constants c^k with |Omega| (c^{k+1}-c^k)/dt = E'_k(g~ - B dphi_hat + C drho)
    B = d.B_block(phi)
    C = d.C_block(rho, s)
    lam = ((gt - B @ dphi_hat + C @ drho_p).reshape(d.K, d.Nc).sum(1)) / d.area_total
    c = np.concatenate([[0.0], np.cumsum(d.dt * lam)])
    dphi_rec = (dphi_hat.reshape(d.K + 1, d.N) + c[:, None]).ravel()
    dphi_rec = ipm.phi_gauge(d, dphi_rec)
    assert np.allclose(dphi_rec, dphi, atol=1e-9)


# ------------------------------------------------- BB preconditioner (Sec. 4.3.3)
@pytest.mark.parametrize("n,K", [(2, 2), (3, 3), (4, 2)])
def test_atilde_is_half_the_galerkin_product_of_A(n, K):
    """With rho constant in time, every A^k uses the edge values R_E rho, and J
    lifts a coarse function to one that jumps only across fine edges lying on
    coarse edges.  Each coarse edge holds two fine edges of half its length
    whose centre distance is also halved (the 4:1 refinement is self-similar),
    and lambda = 1/2 on both meshes, so J^T A^k J = 2 A~^k exactly."""
    d = ipm.discretise(n, K)
    rng = np.random.default_rng(10 * n + K)
    rc = rng.uniform(0.5, 2, d.Nc)
    A = d.A_block(np.tile(rc, K), rc, rc)
    JJ = d.J_block(K + 1)
    G = (JJ.T @ A @ JJ).toarray()
    At = d.A_tilde_block(np.tile(rc, K)).toarray()
    Nc = d.Nc
    for k in range(K):
        blk = slice(k * Nc, (k + 1) * Nc)
        assert np.abs(0.5 * G[blk, blk] - At[blk, blk]).max() < 1e-13 * np.abs(At).max()


@pytest.mark.parametrize("n,K", [(2, 3), (3, 3)])
def test_atilde_slice_k_depends_on_rho_k_alone(n, K):
    """Sec. 4.3.3 builds A~^k from rho^k only.  With rho varying in time, the k-th
    block of A~ must equal half the Galerkin product J^T A J of a fine Laplacian
    whose edge densities come from rho^k alone (the constant-in-time identity above
    applied to each slice on its own), and no other slice of rho may move it."""
    d = ipm.discretise(n, K)
    rng = np.random.default_rng(20 * n + K)
    rho = rng.uniform(0.5, 2, K * d.Nc)
    R = rho.reshape(K, d.Nc)
    At = d.A_tilde_block(rho).toarray()
    J1 = d.J_block(1)
    Nc = d.Nc
    for k in range(K):
        Ak = d.A_block(np.tile(R[k], K), R[k], R[k]).tocsr()[: d.N, : d.N]  # slice 1, built from rho^k alone
        G = (J1.T @ Ak @ J1).toarray()
        blk = slice(k * Nc, (k + 1) * Nc)
        assert np.abs(0.5 * G - At[blk, blk]).max() < 1e-13 * np.abs(At).max(), k
        other = rho.copy().reshape(K, Nc)
        other[np.arange(K) != k] *= rng.uniform(0.5, 2, (K - 1, Nc))
        At2 = d.A_tilde_block(other.ravel()).toarray()
        assert np.abs(At2[blk, blk] - At[blk, blk]).max() == 0.0, k


@pytest.mark.parametrize("n,K", [(2, 2), (3, 3)])
def test_btilde_is_the_block_transpose_of_B_on_coarse_functions(n, K):
    """Reading R5 with R_T = R_E^T diag(|w||e|) and lambda = 1/2 gives
    J^T R_f^T W = R_T, so on coarse functions B~ carries the same transport
    term (grad phi^j . grad, averaged over the two density slices next to
    phi^j) as B, on the swapped time staggering: block (j, k) of J^T B~ equals
    block (k, j) of B J except for the time differences, which enter the two
    with opposite signs, (J^T B~)_{jk} - (B J)_{kj} = (2/dt) M' (d_jk - d_{j,k+1})."""
    d = ipm.discretise(n, K)
    phi = np.random.default_rng(n + K).standard_normal((K + 1) * d.N)
    JJ = d.J_block(K + 1)
    L = (JJ.T @ d.B_tilde_block(phi)).toarray()
    R = (d.B_block(phi) @ JJ).toarray()
    Nc, Mp = d.Nc, d.Mc.toarray()
    scale = np.abs(L).max()
    for j in range(K + 1):
        for k in range(K):
            diff = L[j * Nc:(j + 1) * Nc, k * Nc:(k + 1) * Nc] - R[k * Nc:(k + 1) * Nc, j * Nc:(j + 1) * Nc]
            want = (2.0 / d.dt) * Mp * (float(j == k) - float(j == k + 1))
            assert np.abs(diff - want).max() < 1e-13 * scale


@pytest.mark.parametrize("geom,n,K", [("tri", 2, 2), ("tri", 3, 3), ("cube", 2, 2)])
def test_exact_bb_application_solves_its_triangular_factor(geom, n, K):
    """With exact inner solves the BB application returns (x, y) with
      * y the solution of the approximated Schur system of Eq. (schur-linear-system),
        P (C - B M^-1 B~ A~^+ M') P^T y = -d for d in the range of P, built here
        with a dense pseudo-inverse instead of the rescaled system (pseudoschur-bis)
        and y = M'^-1 A~ z that the application uses;
      * y in the range of P^T, as Sec. 4.3.3 requires of the solution;
      * x from the first block row of the projected system, A x = c - B^T P^T y
        up to per-slice constants (the range of A), with zero slice means.
    On triangles and on the cube grid of the 3D variant."""
    d = _disc(geom, n, K)
    rng = np.random.default_rng(40 + n + K)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    phi = 0.3 * rng.standard_normal((K + 1) * d.N)
    rho = ipm.renormalise(d, rng.uniform(0.5, 2, K * d.Nc), r0)
    s = rng.uniform(0.5, 2, K * d.Nc)
    Np, Nr = (K + 1) * d.N, K * d.Nc
    P = d.P_block().toarray()
    c = rng.standard_normal(Np)
    dv = P @ rng.standard_normal(Nr)
    x, y = ops.bb_apply_exact(d, phi, rho, s, r0, r1, np.concatenate([c, dv]))
    Mp = d.Mc_block().toarray()
    Minv = np.diag(1.0 / np.tile(d.t.fine.area, K + 1))
    B = d.B_block(phi).toarray()
    St = P @ (d.C_block(rho, s).toarray()
              - B @ Minv @ d.B_tilde_block(phi).toarray() @ np.linalg.pinv(d.A_tilde_block(rho).toarray()) @ Mp) @ P.T
    assert np.abs(St @ y + dv).max() < 1e-9 * np.abs(dv).max()
    # y = M'^-1 A~ z has zero mass per slice (A~ has zero column sums), so P^T y = y
    assert np.abs(P.T @ y - y).max() < 1e-12 * np.abs(y).max()
    Kp = d.projected_kkt(phi, rho, s, r0, r1).toarray()
    r = (Kp[:Np] @ np.concatenate([x, y]) - c).reshape(K + 1, d.N)
    assert np.abs(r - r.mean(axis=1, keepdims=True)).max() < 1e-10 * np.abs(c).max()
    assert np.abs(x.reshape(K + 1, d.N).mean(axis=1)).max() < 1e-12 * np.abs(x).max()


@pytest.mark.parametrize("geom,n,K", [("tri", 2, 2), ("tri", 3, 3), ("cube", 2, 3)])
def test_simple_application_inverts_its_block_approximation(geom, n, K):
    """The three SIMPLE factors (Sec. 4.2) multiply to the inverse of the projected
    system with A replaced by Diag(A): u = (x, y) solves
    [Diag(A), B^T P^T; P B, -P C P^T] u = (c; d) for d in the range of P,
    checked against that matrix assembled from the projected system's blocks."""
    d = _disc(geom, n, K)
    rng = np.random.default_rng(60 + n + K)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    phi = 0.3 * rng.standard_normal((K + 1) * d.N)
    rho = ipm.renormalise(d, rng.uniform(0.5, 2, K * d.Nc), r0)
    s = rng.uniform(0.5, 2, K * d.Nc)
    Np = (K + 1) * d.N
    P = d.P_block()
    c = rng.standard_normal(Np)
    dv = P @ rng.standard_normal(K * d.Nc)
    x, y = ops.simple_apply_exact(d, phi, rho, s, r0, r1, np.concatenate([c, dv]))
    Kp = d.projected_kkt(phi, rho, s, r0, r1).toarray()
    Kp[:Np, :Np] = np.diag(np.diag(Kp[:Np, :Np]))
    r = Kp @ np.concatenate([x, y]) - np.concatenate([c, dv])
    assert np.abs(r).max() < 1e-10 * max(np.abs(c).max(), np.abs(dv).max())
    assert np.abs(P.T @ y - y).max() < 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("geom,n,K", [("tri", 2, 3), ("tri", 4, 5), ("cube", 3, 4)])
def test_simple_schur_complement_is_its_time_lines_without_potential_gradient(geom, n, K):
    """SIMPLE's Schur complement -S^ = P C P^T + P B A^-1 B^T P^T (Sec. 4.2, A^ =
    Diag(A)) couples only the slices of one coarse cell when the potential has no
    spatial gradient: it is then P L P^T with L block tridiagonal in time per
    coarse cell C, diagonal |C| s^k/rho^k + w^k_C + w^{k+1}_C and couplings
    -w^{k+1}_C, w^j_C = sum over the fine cells f of C of |f|^2 / (A^_{j,f} dt^2).
    This is the operator whose exact inverse on the zero-slice-sum subspace
    preconditions the GPU's inner SIMPLE solve.  A potential varying in space
    adds couplings between cells, so the two then differ."""
    d = _disc(geom, n, K)
    rng = np.random.default_rng(40 + n + K)
    r0 = rng.uniform(0.5, 2, d.Nc)
    r1 = rng.uniform(0.5, 2, d.Nc)
    r1 *= (d.t.coarse.area @ r0) / (d.t.coarse.area @ r1)
    rho = ipm.renormalise(d, rng.uniform(0.5, 2, K * d.Nc), r0)
    s = rng.uniform(0.5, 2, K * d.Nc)
    P = d.P_block()

    def neg_schur(phi):
        Ad = d.A_block(rho, r0, r1).diagonal()
        Bp = (P @ d.B_block(phi)).tocsr()
        return (P @ d.C_block(rho, s) @ P.T + Bp @ sp.diags(1.0 / Ad) @ Bp.T).toarray(), Ad

    def time_lines(Ad):
        f2 = d.t.fine.area ** 2 / d.dt ** 2
        w = np.array([d.J.T @ (f2 / Ad[j * d.N:(j + 1) * d.N]) for j in range(K + 1)])   # (K+1) x N'
        cdiag = (np.tile(d.t.coarse.area, K) * s / rho).reshape(K, d.Nc)
        L = sp.diags((cdiag + w[:-1] + w[1:]).ravel())
        if K > 1:
            off = -w[1:-1].ravel()
            L = L + sp.diags(off, d.Nc) + sp.diags(off, -d.Nc)
        return (P @ L @ P.T).toarray()

    flat = np.repeat(rng.standard_normal(K + 1), d.N)          # constant in space on every slice
    S, Ad = neg_schur(flat)
    T = time_lines(Ad)
    assert np.abs(S - T).max() < 1e-12 * np.abs(S).max()
    wavy = 0.3 * rng.standard_normal((K + 1) * d.N)
    S, Ad = neg_schur(wavy)
    assert np.abs(S - time_lines(Ad)).max() > 1e-3 * np.abs(S).max()


def _gmres_right(apply_op, b, apply_prec, tol=1e-5, maxit=300):
    """Iterations of right-preconditioned GMRES (dense, two Gram-Schmidt passes) to ||r|| <= tol ||b||."""
    beta = np.linalg.norm(b)
    V = np.zeros((maxit + 1, b.size))
    H = np.zeros((maxit + 1, maxit))
    V[0] = b / beta
    for j in range(maxit):
        w = apply_op(apply_prec(V[j]))
        for _ in range(2):
            h = V[:j + 1] @ w
            w = w - h @ V[:j + 1]
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2)
        e1[0] = beta
        yk = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        if np.linalg.norm(H[:j + 2, :j + 1] @ yk - e1) <= tol * beta or H[j + 1, j] < 1e-14 * beta:
            return j + 1
        V[j + 1] = w / H[j + 1, j]
    return maxit


@pytest.mark.slow
def test_preconditioner_iteration_trends_along_the_barrier_path():
    """Sec. 4.2-4.3 and the summary of Sec. 4.4, with exact inner solves: at the
    first Newton step of each mu stage (4x4 squares, K = 4, the 3-Gaussian
    mixtures of seeds 2 and 3, floor 1e-4), the BB-preconditioned GMRES needs
    more iterations as mu decreases, while SIMPLE needs fewer over the late
    stages and more than BB at mu = 1 (measured: BB 4 -> 18, SIMPLE 56 -> 26)."""
    from ot_inputs import mixture_params

    n, K = 4, 4
    d = ipm.discretise(n, K)
    r0 = make_density(n, *mixture_params(2, 3), 1e-4)
    r1 = make_density(n, *mixture_params(3, 3), 1e-4)
    opt = ipm.IPMOptions()
    phi, rho, s = ipm.initial_point(d, r0, r1, opt.mu0)
    mu = opt.mu0
    Np = (K + 1) * d.N
    bb_its, simple_its = [], []
    for _ in range(ipm.stage_count(K, opt, d.area_total)):
        F = ipm.residual(d, phi, rho, s, r0, r1, mu)
        f0 = fn = ipm.residual_norm(F)
        first = True
        while fn > opt.newton_tol * max(1.0, f0):
            if first:
                Kp = d.projected_kkt(phi, rho, s, r0, r1)
                gt = -F[1] + np.tile(d.t.coarse.area, K) * F[2] / rho
                b = np.concatenate([-F[0], d.P_block() @ gt])
                state = (phi, rho, s, r0, r1)
                bb_its.append(_gmres_right(lambda x: Kp @ x, b,
                                           lambda v: np.concatenate(ops.bb_apply_exact(d, *state, v))))
                simple_its.append(_gmres_right(lambda x: Kp @ x, b,
                                               lambda v: np.concatenate(ops.simple_apply_exact(d, *state, v))))
                first = False
            dphi, drho, ds, _ = ipm.newton_direction(d, phi, rho, s, r0, r1, mu)
            a = min(ipm.step_length(rho, drho, opt.tau), ipm.step_length(s, ds, opt.tau))
            phi, rho, s = phi + a * dphi, ipm.renormalise(d, rho + a * drho, r0), s + a * ds
            F = ipm.residual(d, phi, rho, s, r0, r1, mu)
            fn = ipm.residual_norm(F)
        mu *= opt.mu_factor
    assert len(bb_its) == 10
    assert all(b1 <= b2 for b1, b2 in zip(bb_its, bb_its[1:])) and bb_its[-1] >= 3 * bb_its[0]
    peak = int(np.argmax(simple_its))
    assert peak <= 2 and all(a >= b for a, b in zip(simple_its[peak:], simple_its[peak + 1:]))
    assert simple_its[-1] < 0.6 * simple_its[peak] and simple_its[0] > 5 * bb_its[0]


# ----------------------------------------------------------------- symmetries
def _image(points, mapped):
    """Index j with points[j] == mapped[i] for every i (a permutation, else AssertionError)."""
    dist = np.linalg.norm(points[None, :, :] - mapped[:, None, :], axis=2)
    j = dist.argmin(axis=1)
    assert dist[np.arange(len(j)), j].max() < 1e-12 and len(set(j.tolist())) == len(j)
    return j


def test_solution_respects_time_reversal_and_mesh_symmetries():
    """The barrier problem is strictly convex in rho (Sec. 3), so its solution inherits
    every symmetry of the data.  Swapping rho_in and rho_f reverses time: rho^k and s^k
    go to slice K+1-k, phi^k to -phi^(K+2-k), the cost is unchanged.  The grid of squares
    cut along their (0,0)->(1,1) diagonals is invariant under the point reflection
    (x, y) -> (1-x, 1-y) and the swap (x, y) -> (y, x), which permute the cells.  Random
    (not symmetric) densities, so any term that treats the two time ends, the two cells
    of an edge or the two axes differently shows up."""
    n, K = 3, 3
    d = ipm.discretise(n, K)
    rng = np.random.default_rng(11)
    area = d.t.coarse.area
    r0, r1 = rng.uniform(0.2, 2.0, d.Nc), rng.uniform(0.2, 2.0, d.Nc)
    r0, r1 = r0 / (area @ r0), r1 / (area @ r1)
    opt = ipm.IPMOptions(gap_tol=1e-3, final_newton_tol=1e-12)

    def solve(a, b):
        res = ipm.ipm_solve(d, a, b, opt)
        return (res.rho.reshape(K, d.Nc), res.s.reshape(K, d.Nc),
                ipm.phi_gauge(d, res.phi).reshape(K + 1, d.N), res.cost)

    rho, s, phi, c = solve(r0, r1)
    scale = np.abs(phi).max()
    # time reversal
    rho2, s2, phi2, c2 = solve(r1, r0)
    assert abs(c2 - c) < 1e-10 * c
    assert np.abs(rho2 - rho[::-1]).max() < 1e-9 * rho.max()
    assert np.abs(s2 - s[::-1]).max() < 1e-9 * s.max()
    assert np.abs(phi2 + phi[::-1]).max() < 1e-9 * scale
    # mesh symmetries
    for f in (lambda p: 1.0 - p, lambda p: p[:, ::-1]):
        pc = _image(d.t.coarse.bary, f(d.t.coarse.bary))
        pf = _image(d.t.fine.bary, f(d.t.fine.bary))
        assert np.allclose(area[pc], area) and np.allclose(d.t.fine.area[pf], d.t.fine.area)
        rho3, s3, phi3, c3 = solve(r0[pc], r1[pc])
        assert abs(c3 - c) < 1e-10 * c
        assert np.abs(rho3 - rho[:, pc]).max() < 1e-9 * rho.max()
        assert np.abs(s3 - s[:, pc]).max() < 1e-9 * s.max()
        assert np.abs(phi3 - phi[:, pf]).max() < 1e-9 * scale
    # the data are not symmetric themselves
    assert np.abs(r0[pc] - r0).max() > 0.1 and np.abs(r1 - r0).max() > 0.1


# ------------------------------------------------------------------- IPM
def test_uniform_densities_exact_solution():
    """rho_in = rho_f = c: rho^k = c, s = mu/c, phi^k = -(k-1) dt mu/c + const, C = 0, one Newton step per stage."""
    n, K, c = 3, 4, 1.0
    d = ipm.discretise(n, K)
    r0 = np.full(d.Nc, c)
    res = ipm.ipm_solve(d, r0, r0.copy(), ipm.IPMOptions(final_newton_tol=1e-12))
    mu = res.mu
    assert all(steps == 1 for _, steps, _ in res.stages)
    assert np.allclose(res.rho, c, rtol=0, atol=1e-13)
    assert np.allclose(res.s, mu / c, rtol=1e-12)
    k = np.arange(K + 1)
    expect = ipm.phi_gauge(d, np.repeat(-k * d.dt * mu / c, d.N))
    assert np.allclose(res.phi, expect, atol=1e-14)
    assert abs(res.cost) < 1e-25
    assert np.isclose(res.cost - res.dual, mu * K / (K + 1), rtol=1e-12)


def test_uniform_densities_exact_solution_on_a_graded_mesh():
    """The same closed form where the coarse cells differ in area.  With phi constant
    in space, J^T M 1 = |c'| and the slack enters F_rho as M' s, so every term of
    F_rho is a multiple of the area vector and rho^k = c, s = mu/c still solve the
    system.  A slack weighted by anything other than the cell areas (1/N', say, which
    equals M' on the uniform grid) leaves a spatially varying F_rho and moves rho."""
    n, K, c = 3, 3, 1.0
    d = _graded_discretisation(n, K)
    assert np.ptp(d.t.coarse.area) > 0.01 and abs(d.area_total - 1.0) < 1e-14
    r0 = np.full(d.Nc, c)
    res = ipm.ipm_solve(d, r0, r0.copy(), ipm.IPMOptions(final_newton_tol=1e-12))
    mu = res.mu
    assert all(steps == 1 for _, steps, _ in res.stages)
    assert np.allclose(res.rho, c, rtol=0, atol=1e-13)
    assert np.allclose(res.s, mu / c, rtol=1e-12)
    k = np.arange(K + 1)
    expect = ipm.phi_gauge(d, np.repeat(-k * d.dt * mu / c, d.N))
    assert np.allclose(res.phi, expect, atol=1e-14)
    assert abs(res.cost) < 1e-25
    assert np.isclose(res.cost - res.dual, mu * d.area_total * K / (K + 1), rtol=1e-12)


def test_mu_schedule_matches_table3():
    """mu <- mu/5 from 1 reproduces every row label of Table 3 and stops after ten stages."""
    labels = [float(x) for x in open(os.path.join(GOLDEN, "mu_schedule_table3.txt")) if x.strip() and x[0] != "#"]
    opt = ipm.IPMOptions()
    assert ipm.stage_count(8, opt) == len(labels) == 10
    mus = [opt.mu0 * opt.mu_factor ** l for l in range(10)]
    for mu, lab in zip(mus, labels):
        assert float(f"{mu:.0e}") == lab


def test_ipm_stops_at_the_first_stage_whose_duality_gap_meets_the_tolerance():
    """The solve stops at the first mu whose barrier solution has C - D <= tol, with
    C and D computed from that solution.  With K = 1 the gap is mu/2, so a rule that
    compares mu itself with tol would run one stage further (tol = 1e-3: 3.2e-4 in
    place of 1.6e-3).  The previous stage's gap comes from its own barrier solution,
    solved alone from the initial point."""
    n, K, tol = 2, 1, 1e-3
    d = ipm.discretise(n, K)
    r0 = make_density(n, [(0.3, 0.3)], [0.15], [1.0], 1e-3)
    r1 = make_density(n, [(0.7, 0.6)], [0.15], [1.0], 1e-3)
    res = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(gap_tol=tol, final_newton_tol=1e-12))
    mus = [m for m, _, _ in res.stages]
    assert len(mus) >= 2 and res.cost - res.dual <= tol
    prev = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(mu0=mus[-2], gap_tol=1e9, final_newton_tol=1e-12))
    assert len(prev.stages) == 1 and prev.mu == mus[-2]
    assert prev.cost - prev.dual > tol


@pytest.fixture(scope="module")
def converged_small():
    n, K = 4, 4
    d = ipm.discretise(n, K)
    r0 = make_density(n, [(0.3, 0.3)], [0.1], [1.0], 1e-3)
    r1 = make_density(n, [(0.7, 0.7)], [0.1], [1.0], 1e-3)
    res = ipm.ipm_solve(d, r0, r1, ipm.IPMOptions(final_newton_tol=1e-12))
    return d, r0, r1, res


def test_duality_gap_identity(converged_small):
    """C - D = mu |Omega| K/(K+1) at a solution (summation by parts of F_phi = 0, F_rho = 0, rho s = mu)."""
    d, r0, r1, res = converged_small
    gap = res.mu * d.area_total * d.K / (d.K + 1)
    assert abs((res.cost - res.dual) - gap) < 1e-9 * gap
    F = ipm.residual(d, res.phi, res.rho, res.s, r0, r1, res.mu)
    assert ipm.residual_norm(F) < 1e-12


@pytest.mark.parametrize("graded", [False, True])
def test_duality_gap_identity_at_any_point(graded):
    """The gap identity off the solution, derived by summation by parts from the
    definitions of F_phi, F_rho (time term J^T M, reading R3), the cost and the
    dual value (reading R15), with R_T = R_E^T diag(|e||w|):
      C - D - mu |Omega| K/(K+1) = dt [ sum_k phi^k.F_phi^k - sum_k rho^k.F_rho^k + sum_k |c'|.(F_s^k) ],
    F_s = rho s - mu.  It holds at every (phi, rho, s), so a term dropped or
    mis-weighted in the residual, the cost or the dual value breaks it; on the
    graded grid |c'| differs from cell to cell."""
    n, K = 3, 4
    d = _graded_discretisation(n, K) if graded else ipm.discretise(n, K)
    phi, rho, s, r0, r1 = _random_state(d, seed=11 + int(graded))
    mu = 0.37
    Fphi, Frho, Fs = ipm.residual(d, phi, rho, s, r0, r1, mu)
    C = ipm.cost(d, phi, rho, r0, r1)
    D = ipm.dual_value(d, phi, r0, r1)
    area = d.t.coarse.area
    rhs = d.dt * (phi @ Fphi - rho @ Frho + np.tile(area, K) @ Fs)
    lhs = C - D - mu * area.sum() * K / (K + 1)
    scale = abs(C) + abs(D) + d.dt * (abs(phi) @ abs(Fphi) + abs(rho) @ abs(Frho))
    assert abs(lhs - rhs) < 1e-13 * scale, (lhs, rhs)


def test_mass_positivity_complementarity(converged_small):
    """Remark one-mass: |c'|^T rho^k = |c'|^T rho^0; rho, s > 0; rho s = mu."""
    d, r0, r1, res = converged_small
    R = res.rho.reshape(d.K, d.Nc)
    assert np.allclose(R @ d.t.coarse.area, d.t.coarse.area @ r0, rtol=0, atol=1e-14)
    assert res.rho.min() > 0 and res.s.min() > 0
    assert np.allclose(res.rho * res.s, res.mu, rtol=1e-9)
    # Newton steps: Sec. 4.1 reports 3-7 per stage and 40-50 in total
    assert 30 <= res.newton_steps <= 60


def test_barycentre_moves_linearly_in_time():
    """Along a W2 geodesic the momentum integral of rho v is constant in time, so the
    centre of mass moves on a straight line at constant speed.  On two-Gaussian
    mixtures the discrete barycentres of rho^k at t_k = k/(K+1) deviate from
    (1 - t_k) b_in + t_k b_f by less than 3% of the displacement at 4x4 squares
    (K = 4) and 0.6% at 8x8 (K = 8), shrinking at least 3x per refinement."""
    dev = []
    for n in (4, 8):
        d = ipm.discretise(n, n)
        c0, s0, w0 = mixture_params(2, 2)
        c1, s1, w1 = mixture_params(3, 2)
        r0 = make_density(n, c0, s0, w0, 1e-3)
        r1 = make_density(n, c1, s1, w1, 1e-3)
        res = ipm.ipm_solve(d, r0, r1)
        R = np.vstack([r0, res.rho.reshape(d.K, d.Nc), r1]) * d.t.coarse.area
        b = R @ d.t.coarse.bary
        t = np.arange(d.K + 2) / (d.K + 1)
        line = (1 - t)[:, None] * b[0] + t[:, None] * b[-1]
        dev.append(np.abs(b - line).max() / np.linalg.norm(b[-1] - b[0]))
    assert dev[0] < 0.03 and dev[1] < 0.006 and dev[1] < dev[0] / 3, dev

@pytest.mark.slow
def test_translation_costs_converge():
    """Translated equal Gaussians: C -> |d|^2/2 along (1,1), where the scheme's effective
    metric is exact; C -> (4/3)|d|^2/2 along x, the walled-strip conductivity 3/4 of this mesh."""
    out = {}
    for n in (4, 8):
        d = ipm.discretise(n, n)
        for name, (c0, c1) in {"diag": ((0.3, 0.3), (0.7, 0.7)), "x": ((0.3, 0.5), (0.7, 0.5))}.items():
            r0 = make_density(n, [c0], [0.1], [1.0], 1e-3)
            r1 = make_density(n, [c1], [0.1], [1.0], 1e-3)
            out[n, name] = ipm.ipm_solve(d, r0, r1).cost
    e_diag = [abs(out[n, "diag"] / 0.16 - 1) for n in (4, 8)]
    e_x = [abs(out[n, "x"] / (0.08 * 4 / 3) - 1) for n in (4, 8)]
    assert e_diag[1] < e_diag[0] < 0.1 and e_diag[1] < 0.03
    assert e_x[1] < e_x[0] < 0.1 and e_x[1] < 0.03


# ----------------------------------------------------------------- adjoint gradient
def _adjoint_case(gap_tol):
    from ot_inputs import mixture_params

    n, K = 3, 3
    d = ipm.discretise(n, K)
    r0 = make_density(n, *mixture_params(1, 2), 1e-2)
    r1 = make_density(n, *mixture_params(51, 2), 1e-2)
    opt = ipm.IPMOptions(gap_tol=gap_tol, final_newton_tol=1e-13)
    return d, r0, r1, opt, ipm.ipm_solve(d, r0, r1, opt)


def test_adjoint_gradient_matches_central_differences():
    """dC/d(rho_in, rho_f) by one transposed-Jacobian solve equals central
    differences of the converged IPM cost along mass-preserving directions
    (h = 1e-6, both runs ending at the same mu with ||F|| <= 1e-13)."""
    from oracle import adjoint

    d, r0, r1, opt, res = _adjoint_case(1e-4)
    g0, g1 = adjoint.cost_gradient(d, res.phi, res.rho, res.s, r0, r1)
    rng = np.random.default_rng(8)
    a = d.t.coarse.area
    h = 1e-6
    for which in (0, 1):
        for _ in range(2):
            v = rng.uniform(-1, 1, d.Nc)
            v -= (a @ v) / a.sum()
            args_p = (r0 + h * v, r1) if which == 0 else (r0, r1 + h * v)
            args_m = (r0 - h * v, r1) if which == 0 else (r0, r1 - h * v)
            fd = (ipm.ipm_solve(d, *args_p, opt).cost - ipm.ipm_solve(d, *args_m, opt).cost) / (2 * h)
            ad = float((g0 if which == 0 else g1) @ v)
            assert abs(fd - ad) <= 1e-6 * abs(fd), (which, fd, ad)


def test_adjoint_gradient_approaches_dual_potential_as_mu_vanishes():
    """The adjoint gradient tends to the envelope form read off the dual value
    (-J^T M phi^1 - dt/4 R_E^T W (grad phi^1)^2 at t = 0, and its mirror at
    t = 1) at rate O(mu): two decades of mu shrink the gap by >= 20x."""
    from oracle import adjoint

    errs = []
    for tol in (1e-4, 1e-6):
        d, r0, r1, opt, res = _adjoint_case(tol)
        g0, g1 = adjoint.cost_gradient(d, res.phi, res.rho, res.s, r0, r1)
        e0, e1 = adjoint.envelope_gradient(d, res.phi)
        errs.append(max(np.linalg.norm(g0 - e0) / np.linalg.norm(g0), np.linalg.norm(g1 - e1) / np.linalg.norm(g1)))
    assert errs[1] < errs[0] / 20 and errs[1] < 1e-3, errs


def test_adjoint_partials_match_finite_differences_of_cost():
    """The explicit partials dC/du and dC/dr (reading R15) against central
    differences of ipm.cost at a random point."""
    from oracle import adjoint

    d = ipm.discretise(2, 2)
    phi, rho, s, r0, r1 = _random_state(d, 9)
    dphi, drho, d0, d1 = adjoint.cost_partials(d, phi, rho, r0, r1)
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(3):
        vp, vr, v0, v1 = (rng.standard_normal(x.size) for x in (phi, rho, r0, r1))
        fd = (ipm.cost(d, phi + h * vp, rho + h * vr, r0 + h * v0, r1 + h * v1)
              - ipm.cost(d, phi - h * vp, rho - h * vr, r0 - h * v0, r1 - h * v1)) / (2 * h)
        an = dphi @ vp + drho @ vr + d0 @ v0 + d1 @ v1
        assert abs(fd - an) < 1e-7 * max(1.0, abs(fd))


@pytest.mark.slow
def test_separable_densities_converge_to_quantile_w2():
    """Densities that vary only in x (a narrow and a wide Gaussian profile with a
    floor, so a dilation as well as a shift): the optimal flow is along x, whose
    cost on this mesh is 4/3 of the Euclidean one (the walled-strip conductivity
    3/4), so C -> (4/3) W2^2 / 2 with W2^2 = int_0^1 |F^-1(u) - G^-1(u)|^2 du from
    the quantile functions of the two profiles (computed here on a fine grid)."""
    from ot_inputs import _split4, coarse_triangles

    c0, s0, c1, s1, floor = 0.4, 0.08, 0.6, 0.15, 1e-2
    prof = lambda x, c, s: floor + np.exp(-(x - c) ** 2 / (2 * s * s))  # noqa: E731

    def cell_average(n, c, s):
        tri = coarse_triangles(n)
        sub = _split4(_split4(tri))
        mids = np.stack([(sub[:, 0] + sub[:, 1]) / 2, (sub[:, 1] + sub[:, 2]) / 2, (sub[:, 2] + sub[:, 0]) / 2], 1)
        v = prof(mids[..., 0], c, s).mean(1).reshape(tri.shape[0], 16).mean(1)
        return v / (0.5 / (n * n) * v.sum())

    x = np.linspace(0.0, 1.0, 400001)
    u = (np.arange(200000) + 0.5) / 200000

    def quantile(c, s):
        f = prof(x, c, s)
        F = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(x))])
        return np.interp(u, F / F[-1], x)

    target = (4.0 / 3.0) * float(np.mean((quantile(c0, s0) - quantile(c1, s1)) ** 2)) / 2.0
    err = {}
    for n in (4, 8):
        d = ipm.discretise(n, n)
        err[n] = ipm.ipm_solve(d, cell_average(n, c0, s0), cell_average(n, c1, s1)).cost / target - 1.0
    assert abs(err[8]) < abs(err[4]) < 0.15 and abs(err[8]) < 0.01, err

