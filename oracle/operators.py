"""Sparse operators of the discrete problem (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Single-slice operators follow Sec. 2.1 of the paper; the space-time block
operators follow Sec. 3 (the blocks of the KKT matrix); the projected system
and the BB approximation follow Sec. 4.3.  Everything is a scipy.sparse
matrix built entry by entry from the definitions; vectors are slice-major:
phi = (phi^1; ...; phi^{K+1}) with N entries per slice, rho and s = (.^1; ...;
.^K) with N' entries per slice.

Readings taken where the paper is silent, ambiguous or inconsistent:
  R3  the time term of F_rho is J^T M (phi^{k+1}-phi^k)/dt, the form that makes
      the Jacobian the symmetric block  [A B^T; B 0]  of Sec. 3.
  R5  G^k maps fine edges to coarse cells; the matrix B~ of Sec. 4.3.2 is read as
        B~ z = -M J D~_t^T z + R_f^T W diag(grad phi) grad J H^T z
      with W = diag(|e| |w|) and R_f the plain average from fine cells to fine
      edges; A~^k = -div' diag(R_E' rho^k) grad' on the coarse mesh.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import TriMesh, TwoLevelMesh


# ---------------------------------------------------------------- one slice
def incidence(m: TriMesh) -> sp.csr_matrix:
    """E: +1 where the cell is the left side of the edge, -1 where it is the right side."""
    ne = m.nedge
    rows = np.concatenate([m.edge_cells[:, 0], m.edge_cells[:, 1]])
    cols = np.concatenate([np.arange(ne), np.arange(ne)])
    vals = np.concatenate([np.ones(ne), -np.ones(ne)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(m.ncell, ne))


def grad(m: TriMesh) -> sp.csr_matrix:
    """Discrete gradient  diag(|w|)^-1 E^T  (Sec. 2.1)."""
    return (sp.diags(1.0 / m.edge_dist) @ incidence(m).T).tocsr()


def div(m: TriMesh) -> sp.csr_matrix:
    """Discrete divergence  -E diag(|e|)  (Sec. 2.1)."""
    return (-incidence(m) @ sp.diags(m.edge_len)).tocsr()


def mass(m: TriMesh) -> sp.dia_matrix:
    return sp.diags(m.area)


def injection(t: TwoLevelMesh) -> sp.csr_matrix:
    """J in R^{N x N'}: J[i, j] = 1 when fine cell i lies in coarse cell j, Eq. (tdens2pot)."""
    N = t.fine.ncell
    return sp.csr_matrix((np.ones(N), (np.arange(N), t.parent)), shape=(N, t.coarse.ncell))


def edge_average(m: TriMesh) -> sp.csr_matrix:
    """Weighted mean from the cells of m to its interior edges (lambda on the left cell)."""
    ne = m.nedge
    rows = np.concatenate([np.arange(ne), np.arange(ne)])
    cols = np.concatenate([m.edge_cells[:, 0], m.edge_cells[:, 1]])
    vals = np.concatenate([m.edge_lambda, 1.0 - m.edge_lambda])
    return sp.csr_matrix((vals, (rows, cols)), shape=(ne, m.ncell))


def recon_edges(t: TwoLevelMesh) -> sp.csr_matrix:
    """R_E: coarse cells -> fine edges, lift by J then average (Sec. 2.1)."""
    return (edge_average(t.fine) @ injection(t)).tocsr()


def recon_cells(t: TwoLevelMesh) -> sp.csr_matrix:
    """R_T = R_E^T diag(|w| |e|): fine edges -> coarse cells (Sec. 2.1)."""
    f = t.fine
    return (recon_edges(t).T @ sp.diags(f.edge_dist * f.edge_len)).tocsr()


def weighted_laplacian(m: TriMesh, edge_coef: np.ndarray) -> sp.csr_matrix:
    """-div diag(edge_coef) grad on mesh m."""
    return (-div(m) @ sp.diags(edge_coef) @ grad(m)).tocsr()


# ---------------------------------------------------------------- blocks
class Discretisation:
    """All single-slice operators of a two-level mesh, plus the time step."""

    def __init__(self, t: TwoLevelMesh, K: int):
        self.t, self.K = t, K
        self.N, self.Nc = t.fine.ncell, t.coarse.ncell
        self.Ne = t.fine.nedge
        self.dt = 1.0 / (K + 1)
        self.M = mass(t.fine)
        self.Mc = mass(t.coarse)
        self.J = injection(t)
        self.grad = grad(t.fine)
        self.div = div(t.fine)
        self.RE = recon_edges(t)
        self.RT = recon_cells(t)
        self.W = t.fine.edge_dist * t.fine.edge_len
        self.area_total = t.coarse.area.sum()

    # slice helpers -------------------------------------------------------
    def phi_slices(self, phi):
        return np.asarray(phi).reshape(self.K + 1, self.N)

    def rho_slices(self, rho):
        return np.asarray(rho).reshape(self.K, self.Nc)

    def rho_ext(self, rho, rho0, rho1):
        """(rho^0, rho^1, ..., rho^K, rho^{K+1}) as a (K+2, N') array."""
        return np.vstack([rho0[None, :], self.rho_slices(rho), rho1[None, :]])

    def rho_tilde(self, rho, rho0, rho1):
        """rho~^k = R_E((rho^k + rho^{k-1})/2) for k = 1..K+1, shape (K+1, Ne)."""
        r = self.rho_ext(rho, rho0, rho1)
        avg = 0.5 * (r[1:] + r[:-1])
        return (self.RE @ avg.T).T

    # block operators -----------------------------------------------------
    def A_block(self, rho, rho0, rho1) -> sp.csr_matrix:
        """A = blkdiag(A^k), A^k = -div diag(rho~^k) grad (Sec. 3)."""
        rt = self.rho_tilde(rho, rho0, rho1)
        return sp.block_diag([weighted_laplacian(self.t.fine, rt[k]) for k in range(self.K + 1)]).tocsr()

    def G_slice(self, phi_k) -> sp.csr_matrix:
        """G^k = R_T diag(grad phi^k), fine edges -> coarse cells (Sec. 3, reading R5)."""
        return (self.RT @ sp.diags(self.grad @ phi_k)).tocsr()

    def B_block(self, phi) -> sp.csr_matrix:
        """B = J^T D_t M + H G D_x (Sec. 3), shape (K N', (K+1) N)."""
        K, dt = self.K, self.dt
        P = self.phi_slices(phi)
        JtM = (self.J.T @ self.M).tocsr()
        blocks = [[None] * (K + 1) for _ in range(K)]
        for k in range(K):
            Gk = self.G_slice(P[k]) @ self.grad
            Gk1 = self.G_slice(P[k + 1]) @ self.grad
            blocks[k][k] = -JtM / dt + 0.5 * Gk
            blocks[k][k + 1] = JtM / dt + 0.5 * Gk1
        for k in range(K):
            for j in range(K + 1):
                if blocks[k][j] is None:
                    blocks[k][j] = sp.csr_matrix((self.Nc, self.N))
        return sp.bmat(blocks).tocsr()

    def C_block(self, rho, s) -> sp.dia_matrix:
        """C = M' diag(rho)^-1 diag(s) (Sec. 3.1)."""
        mc = np.tile(self.t.coarse.area, self.K)
        return sp.diags(mc * np.asarray(s) / np.asarray(rho))

    def Mc_block(self) -> sp.dia_matrix:
        return sp.diags(np.tile(self.t.coarse.area, self.K))

    def M_block(self) -> sp.dia_matrix:
        return sp.diags(np.tile(self.t.fine.area, self.K + 1))

    def J_block(self, slices: int) -> sp.csr_matrix:
        return sp.block_diag([self.J] * slices).tocsr()

    # projected system (Sec. 4.3.1) ---------------------------------------
    def P_block(self) -> sp.csr_matrix:
        """P = I - M' E'^T E' / |Omega|, with E' summing each slice."""
        mc = self.t.coarse.area
        Pk = sp.identity(self.Nc) - sp.csr_matrix(np.outer(mc, np.ones(self.Nc)) / self.area_total)
        return sp.block_diag([Pk] * self.K).tocsr()

    def projected_kkt(self, phi, rho, s, rho0, rho1) -> sp.csr_matrix:
        """[A, B^T P^T; P B, -P C P^T], Eq. (newton-linsys-shift-reduced-projected)."""
        A = self.A_block(rho, rho0, rho1)
        B = self.B_block(phi)
        C = self.C_block(rho, s)
        P = self.P_block()
        return sp.bmat([[A, B.T @ P.T], [P @ B, -(P @ C @ P.T)]]).tocsr()

    # BB preconditioner pieces (Sec. 4.3.2, reading R5) --------------------
    def A_tilde_block(self, rho) -> sp.csr_matrix:
        """A~ = blkdiag(-div' diag(R_E' rho^k) grad') on the coarse mesh."""
        c = self.t.coarse
        Rc = edge_average(c)
        R = self.rho_slices(rho)
        return sp.block_diag([weighted_laplacian(c, Rc @ R[k]) for k in range(self.K)]).tocsr()

    def B_tilde_block(self, phi) -> sp.csr_matrix:
        """B~ (reading R5), shape ((K+1) N, K N'): a fine-mesh (d/dt + grad phi . grad) scaled by M."""
        K, dt = self.K, self.dt
        P = self.phi_slices(phi)
        MJ = (self.M @ self.J).tocsr()
        Rf = edge_average_plain(self.t.fine)
        blocks = [[None] * K for _ in range(K + 1)]
        for j in range(K + 1):
            # spatial part acts on the time average (z^{j-1} + z^j)/2 (H^T)
            S = (Rf.T @ sp.diags(self.W * (self.grad @ P[j])) @ self.grad @ self.J).tocsr()
            if j - 1 >= 0:   # coefficient of z^{j-1}
                blocks[j][j - 1] = -MJ / dt + 0.5 * S
            if j <= K - 1:   # coefficient of z^j
                blocks[j][j] = MJ / dt + 0.5 * S
        for j in range(K + 1):
            for k in range(K):
                if blocks[j][k] is None:
                    blocks[j][k] = sp.csr_matrix((self.N, self.Nc))
        return sp.bmat(blocks).tocsr()

    def schur_bb(self, phi, rho, s) -> sp.csr_matrix:
        """Diag(s) A~ - Diag(rho) B M^-1 B~, the matrix of Eq. (pseudoschur-bis)."""
        B = self.B_block(phi)
        Minv = sp.diags(1.0 / np.tile(self.t.fine.area, self.K + 1))
        return (sp.diags(np.asarray(s)) @ self.A_tilde_block(rho)
                - sp.diags(np.asarray(rho)) @ B @ Minv @ self.B_tilde_block(phi)).tocsr()


def edge_average_plain(m: TriMesh) -> sp.csr_matrix:
    """Unweighted mean (1/2, 1/2) from cells to interior edges."""
    ne = m.nedge
    rows = np.concatenate([np.arange(ne), np.arange(ne)])
    cols = np.concatenate([m.edge_cells[:, 0], m.edge_cells[:, 1]])
    return sp.csr_matrix((np.full(2 * ne, 0.5), (rows, cols)), shape=(ne, m.ncell))


def bb_apply_exact(d: Discretisation, phi, rho, s, rho0, rho1, v):
    """One application of the BB block-triangular preconditioner (Sec. 4.3.3,
    Eq. triang with the Schur block of Eq. pseudoschur-bis) with exact solves:

        z = (Diag(s) A~ - Diag(rho) B M^-1 B~)^-1 (-Diag(rho) d),
        y = M'^-1 A~ z,
        b = c - B^T P^T y, with each slice's mean removed (the range of A^j),
        x^j = the zero-mean solution of A^j x^j = b^j, j = 1..K+1,

    for v = (c; d).  Returns (x, y)."""
    Np = (d.K + 1) * d.N
    v = np.asarray(v, dtype=np.float64)
    c, dv = v[:Np], v[Np:]
    z = spla.spsolve(d.schur_bb(phi, rho, s).tocsc(), -np.asarray(rho) * dv)
    y = (d.A_tilde_block(rho) @ z) / np.tile(d.t.coarse.area, d.K)
    b = (c - d.B_block(phi).T @ (d.P_block().T @ y)).reshape(d.K + 1, d.N)
    rt = d.rho_tilde(rho, rho0, rho1)
    x = np.empty_like(b)
    for j in range(d.K + 1):
        bj = b[j] - np.mean(b[j])
        Aj = weighted_laplacian(d.t.fine, rt[j]).tocsc()
        xj = np.zeros(d.N)
        xj[1:] = spla.spsolve(Aj[1:, :][:, 1:].tocsc(), bj[1:])   # ground one potential: A^j is singular
        x[j] = xj - np.mean(xj)
    return x.ravel(), y


def simple_apply_exact(d: Discretisation, phi, rho, s, rho0, rho1, v):
    """One application of the SIMPLE preconditioner (Sec. 4.2) to the projected
    system (B -> P B, C -> P C P^T), with A^ = Diag(A) and an exact solve of
    S^ = -(P C P^T + P B A^-1 B^T P^T):

        x1 = A^-1 c,   y = S^-1 (d - P B x1),   x = x1 - A^-1 B^T P^T y,

    the product of the three block factors applied to v = (c; d).  S^ is block
    tridiagonal in time and vanishes on per-slice constants; d - P B x1 has zero
    slice sums (it lies in the range of P), and y is the solution with
    |c'|^T y^k = 0 (the range of P^T), found from the system bordered by those
    K constraints.  Returns (x, y)."""
    Np = (d.K + 1) * d.N
    v = np.asarray(v, dtype=np.float64)
    c, dv = v[:Np], v[Np:]
    Ad = d.A_block(rho, rho0, rho1).diagonal()
    P = d.P_block()
    Bp = (P @ d.B_block(phi)).tocsr()
    S = -(P @ d.C_block(rho, s) @ P.T + Bp @ sp.diags(1.0 / Ad) @ Bp.T)
    Y = sp.kron(sp.identity(d.K), sp.csr_matrix(d.t.coarse.area[:, None]))
    bordered = sp.bmat([[S, Y], [Y.T, None]]).tocsc()
    x1 = c / Ad
    y = spla.spsolve(bordered, np.concatenate([dv - Bp @ x1, np.zeros(d.K)]))[:d.K * d.Nc]
    return x1 - (Bp.T @ y) / Ad, y
