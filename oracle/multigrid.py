"""hp-multigrid pieces on explicit matrices (oracle, test infrastructure).

Sec. 5.4 ("Matrix-free preconditioners"): the viscous operator is
preconditioned by a multigrid V-cycle that first lowers the polynomial degree,
then coarsens the mesh (h-levels obtained by refining a coarse grid), with a
direct solve on the coarsest level below 2000 unknowns, FP32 arithmetic inside
the preconditioner and FP64 on the coarse level, and a Chebyshev-accelerated
Jacobi smoother built from the inverse diagonal of each level operator. The
viscosity is stored at each level's quadrature points.

Readings (the paper does not print these details):
* p-sequence k -> 2 -> 1 (then h-levels of degree 1), coarsest level = the
  first with fewer than 2000 unknowns or that cannot be halved.
* Prolongation = embedding (interpolate the coarse polynomial at the fine
  nodes); restriction = its transpose.
* Chebyshev(degree d) on D^-1 A with eigenvalue interval [lmax/20, lmax],
  lmax = 1.2 * (largest eigenvalue estimate), the textbook three-term
  recurrence (Saad 2003, Alg. 12.1 applied to the Jacobi-preconditioned system).
* One pre- and one post-smoothing application per level; zero initial guess
  for the pre-smoother.
* Linearization velocity on a coarse level = interpolation of the fine field
  at the coarse Gauss-Lobatto nodes; a coarse node on an interface between
  two children is taken from the child with the lower index.
* Viscosity on the levels (Sec. 5.4: the quadrature-point data of all levels
  is updated through the transfer operators): the analytic field is evaluated
  at each level's points; Carreau-Yasuda from the interpolated velocity; the
  cellwise-constant sphere field is carried down by the transfer of
  piecewise constants - the same value on a p-level, the mean of the eight
  children on an h-level (its L2 projection). Re-evaluating the sphere field
  with each level's coarser Gauss rule instead gives levels that disagree and
  a V-cycle that stalls at high contrast (a test keeps that comparison).
Pinned in tests: prolongation reproduces coarse polynomials exactly;
restriction equals the transpose; the smoother's error propagation equals the
closed-form scaled Chebyshev polynomial on eigenvectors. The V-cycle as a whole
is "parity unpinned" against the paper.
"""
import numpy as np
import scipy.sparse as sp

from . import basis, quadrature


def level_sequence(mesh, k, ncomp, coarse_threshold=2000):
    """[(mesh, degree), ...] fine to coarse."""
    levels = [(mesh, k)]
    for kk in ([2, 1] if k > 2 else ([1] if k == 2 else [])):
        levels.append((mesh, kk))
    m = mesh
    while levels[-1][0].n_cells * ncomp * (levels[-1][1] + 1) ** 3 >= coarse_threshold:
        try:
            m = levels[-1][0].coarsen()
        except ValueError:
            break
        levels.append((m, levels[-1][1]))
    return levels


def p_embedding_1d(k_fine, k_coarse):
    """E[i, j] = l^coarse_j(xi^fine_i)."""
    xf, _ = quadrature.gauss_lobatto(k_fine + 1)
    xc, _ = quadrature.gauss_lobatto(k_coarse + 1)
    return basis.lagrange_values(xc, xf)


def h_embedding_1d(k):
    """[E0, E1]: child c covers [c/2, (c+1)/2] of the parent, E_c[i, j] = l_j((xi_i + c)/2)."""
    x, _ = quadrature.gauss_lobatto(k + 1)
    return [basis.lagrange_values(x, 0.5 * (x + c)) for c in (0, 1)]


def prolongation_p(mesh, k_fine, k_coarse, ncomp):
    E = p_embedding_1d(k_fine, k_coarse)
    cell = np.kron(np.eye(ncomp), np.kron(E, np.kron(E, E)))  # z slowest
    return sp.block_diag([cell] * mesh.n_cells, format='csr')


def prolongation_h(mesh_fine, mesh_coarse, k, ncomp):
    Es = h_embedding_1d(k)
    n3 = (k + 1) ** 3
    mf = ncomp * n3
    rows, cols, vals = [], [], []
    for ef in range(mesh_fine.n_cells):
        i, j, l = mesh_fine.cell_ijk(ef)
        ec = mesh_coarse.cell_index((i // 2, j // 2, l // 2))
        blk = np.kron(Es[l % 2], np.kron(Es[j % 2], Es[i % 2]))
        full = np.kron(np.eye(ncomp), blk)
        r, c = np.nonzero(np.ones_like(full))
        rows.append(ef * mf + r)
        cols.append(ec * mf + c)
        vals.append(full.ravel())
    N_f, N_c = mesh_fine.n_cells * mf, mesh_coarse.n_cells * mf
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N_f, N_c)).tocsr()


def interpolate_down_p(u_fine, mesh, k_fine, k_coarse, ncomp):
    """Coarse nodal values = fine polynomial at the coarse nodes (same cells)."""
    xf, _ = quadrature.gauss_lobatto(k_fine + 1)
    xc, _ = quadrature.gauss_lobatto(k_coarse + 1)
    I1 = basis.lagrange_values(xf, xc)
    cell = np.kron(np.eye(ncomp), np.kron(I1, np.kron(I1, I1)))
    U = np.asarray(u_fine).reshape(mesh.n_cells, -1)
    return (U @ cell.T).reshape(-1)


def interpolate_down_h(u_fine, mesh_fine, mesh_coarse, k, ncomp):
    x, _ = quadrature.gauss_lobatto(k + 1)
    n = k + 1
    child = (x > 0.5).astype(int)          # ties (x == 0.5) go to child 0
    local = 2.0 * x - child
    Ufine = np.asarray(u_fine).reshape(mesh_fine.n_cells, ncomp, n, n, n)
    out = np.zeros((mesh_coarse.n_cells, ncomp, n, n, n))
    L = basis.lagrange_values(x, local)    # L[j, i] = l_i(local_j)
    for ec in range(mesh_coarse.n_cells):
        ci, cj, cl = mesh_coarse.cell_ijk(ec)
        for jz in range(n):
            for jy in range(n):
                for jx in range(n):
                    ef = mesh_fine.cell_index((2 * ci + child[jx], 2 * cj + child[jy], 2 * cl + child[jz]))
                    w = np.einsum('z,y,x->zyx', L[jz], L[jy], L[jx])
                    out[ec, :, jz, jy, jx] = np.einsum('czyx,zyx->c', Ufine[ef], w)
    return out.reshape(-1)


def level_viscosity(levels, rheology, u=None):
    """[(nu_cell, nu_face)] per level (fine to coarse), per the readings above."""
    from .sipg import SIPG
    out, discs, u_l = [], [], u
    for l, (m, k) in enumerate(levels):
        S = SIPG(m, k, 3)
        if l > 0:
            Fm, Fk = levels[l - 1]
            if rheology['law'] == 'carreau':
                u_l = (interpolate_down_p(u_l, m, Fk, k, 3) if Fm.n_cells == m.n_cells
                       else interpolate_down_h(u_l, Fm, m, k, 3))
            if rheology['law'] == 'sinker' and rheology.get('projection', 'cell') == 'cell':
                fine = out[-1][0][:, 0]
                if Fm.n_cells == m.n_cells:
                    v = fine.copy()
                else:
                    v = np.zeros(m.n_cells)
                    for ef in range(Fm.n_cells):
                        i, j, kk = Fm.cell_ijk(ef)
                        v[m.cell_index((i // 2, j // 2, kk // 2))] += fine[ef] / 8.0
                out.append((np.repeat(v[:, None], S.nq ** 3, 1),
                            np.repeat(v[:, None, None], 6, 1).repeat(S.nq ** 2, 2)))
                continue
        out.append(S.viscosity_at_points(rheology, u_l))
    return out


def inverse_diagonal(A):
    return 1.0 / A.diagonal()


def chebyshev(A, dinv, b, x0, degree, lmin, lmax):
    """Chebyshev-accelerated Jacobi: degree steps of the three-term recurrence."""
    op = A if callable(A) else (lambda v: A @ v)
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    x = np.array(x0, dtype=np.float64)
    rho = 1.0 / sigma
    r = b - op(x)
    d = dinv * r / theta
    x = x + d
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = b - op(x)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        x = x + d
        rho = rho_new
    return x


def chebyshev_error_polynomial(lam, degree, lmin, lmax):
    """Closed form T_d((theta - lam)/delta) / T_d(theta/delta) of the smoother."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    T = np.polynomial.chebyshev.Chebyshev.basis(degree)
    return T((theta - lam) / delta) / T(theta / delta)


def lanczos_lmax(A, dinv, v0, steps):
    """Largest Ritz value of D^-1 A after `steps` Lanczos steps (D-inner product)."""
    op = A if callable(A) else (lambda v: A @ v)
    # symmetric form: B = D^-1/2 A D^-1/2
    s = np.sqrt(dinv)
    q = v0 / np.linalg.norm(v0)
    q_prev = np.zeros_like(q)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = s * op(s * q) - beta * q_prev
        alpha = q @ w
        w -= alpha * q
        alphas.append(alpha)
        beta = np.linalg.norm(w)
        if beta == 0.0:
            break
        betas.append(beta)
        q_prev, q = q, w / beta
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:m - 1], 1) + np.diag(betas[:m - 1], -1)
    return np.linalg.eigvalsh(T)[-1]


class VCycle:
    """Reference V-cycle on explicit level matrices (FP64)."""

    def __init__(self, mats, prolongations, degree=3, lmax=None, smoothing_range=20.0):
        self.A = mats                      # fine to coarse
        self.P = prolongations             # P[l] maps level l+1 -> level l
        self.dinv = [inverse_diagonal(A) for A in mats]
        self.degree = degree
        self.lmax = lmax
        self.range = smoothing_range
        self.coarse = mats[-1].toarray() if hasattr(mats[-1], 'toarray') else np.asarray(mats[-1])

    def __call__(self, b, level=0):
        A = self.A[level]
        if level == len(self.A) - 1:
            return np.linalg.solve(self.coarse, b)
        lmax = self.lmax[level]
        lmin = lmax / self.range
        x = chebyshev(A, self.dinv[level], b, np.zeros_like(b), self.degree, lmin, lmax)
        r = b - A @ x
        xc = self(self.P[level].T @ r, level + 1)
        x = x + self.P[level] @ xc
        x = chebyshev(A, self.dinv[level], b, x, self.degree, lmin, lmax)
        return x
