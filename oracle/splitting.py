"""One time step of the dual splitting (projection) scheme (oracle, test infrastructure).

Sec. 3.2 / 5.1 / 5.4, Alg. 1 of the paper, with the convective term explicit
(alpha_c = 0), on grids of affine hexahedra (oracle.mesh: the box, the
backward-facing-step channel) whose Dirichlet faces carry velocity data g per
boundary id (constant vectors: no-slip walls, the moving lid of a cavity; or
functions of the position: the inflow profile, optionally ramped in time), and
whose outflow faces are velocity Neumann (traction free) with p = 0. Every form below is evaluated element by element
with explicit basis functions at the Gauss points, as written in the paper:

* BDF-m and extrapolation coefficients (textbook values, "see Hairer1993";
  READING: BDF1 = (1; 1; 1), BDF2 = (3/2; 2, -1/2; 2, -1); the first step of a
  run uses BDF1, then BDF2 - "sequentially increasing the order").
* Convective term, Eq. (convective_term_weak), w = u:
      c_h(v, u; w) = (v, (w.grad) u)_e - (v, ({{w}}.n) u)_de + (v, ({{w}}.n) u^dag)_de,
      u^dag = {{u}} + 1/2 sign({{w}}.n) [u],   [u] = u^- - u^+,
  with the mirror principle on Dirichlet faces (u^+ = -u^- + 2g, and w^+ alike).
* Convective step, Eq. (convective_step_weak):
      (gamma0/dt) M uhat = M b + sum_i (alpha_i/dt) M u^{n-i} - sum_i beta_i C(u^{n-i}).
  READING: the body force b is given by its interpolant b_h in the velocity space.
* Pressure step, Eq. (pressure_step_weak): the SIPG Laplacian (oracle.sipg)
  against the right-hand side
      (gamma0/dt) [ (grad q, uhat)_e - (q, {{uhat}}.n)_de ]
  where on Dirichlet faces {{uhat}} = g_uhat of Eq. (guhat_consistent_BC) and the
  Neumann datum h_p of Eq. (pressure_Neumann_BC) enters as +(q, h_p)_GammaD
  (the average normal gradient of the mirrored pressure equals h_p). Hence on a
  Dirichlet face the integrand is  h_p - (gamma0/dt) g_uhat.n.
      g_uhat = (dt/gamma0) b - (dt/gamma0) sum_{i<m} beta_i (u^{n-i}.grad)u^{n-i}
               + sum_{i<m} (alpha_i/gamma0) g
      h_p = n.b - n.d_t g - sum_{i<m_p} betabar_i n.(u^{n-i}.grad)u^{n-i}
            - nu^dd n.(curl omega^dd) + 2 n.(eps(u^dd) grad nu^dd)
  with m_p = min(m - 1, 2), u^dd = sum_{i<m_p} betabar_i u^{n-i} (betabar the
  extrapolation coefficients of order m_p), nu^dd = eta(gamma_dot(eps(u^dd)))
  pointwise, omega^dd the element-local L2 projection of curl u^dd onto Q_k
  (Sec. 5.1, vorticity projection of Alg. 1). d_t g = 0 (steady data; the
  paper's BDF approximation of d_t g gives exactly 0 for constant g).
  READINGS: (i) the convective sum in h_p is written with beta_i but runs to
  m_p - 1; the order-m_p coefficients betabar_i are taken (consistent
  extrapolation); (ii) grad nu^dd is the gradient of the element-local L2
  projection of nu^dd onto Q_k (the paper does not say how it is formed; the
  same mechanism as the vorticity); (iii) the traces in h_p and g_uhat are the
  interior (own cell) traces.
  The pure-Neumann pressure problem (velocity Dirichlet on every wall) is made
  solvable by a mean-free right-hand side and solved for the mean-free
  solution (Sec. 3.2).
* Projection step, Eq. (projection_step_weak):
      (gamma0/dt) M uhathat = (gamma0/dt) M uhat + (div v, p)_e - (v, {{p}} n)_de,
  {{p}} = p^- on velocity-Dirichlet (pressure-Neumann) faces.
* Viscous step, Eq. (viscous_step_weak) with alpha_c = 0:
      ((gamma0/dt) M + A(nu)) u^{n+1} = (gamma0/dt) M uhathat + D(g, nu),
  D the Dirichlet data terms of the SIPG viscous form (mirror u^+ = -u^- + 2g):
      D_a = -(2 nu eps(phi_a) n, g)_GammaD + (2 tau, phi_a.g + (phi_a.n)(g.n))_GammaD.
  nu "linear implicit" = eta(gamma_dot(eps(u^#))), u^# = sum_{i<m} beta_i u^{n-i}
  (Alg. 1 then leaves its loop after one pass), or "implicit" by the
  Picard/Aitken loop of oracle.nonlinear.
  With alpha_c = 1 and u* = u^# (the linearly implicit convective term of
  Eq. viscous_step_with_convection) the operator gains c_h(v, u; u^#) - not
  symmetric - and the right-hand side sum_i beta_i c_h(v, u^{n-i}; u^{n-i})
  (``convective_blocks``, ``convective_wall_rhs``).
* Time step, Eq. (CFL_timestep_selection): dt = Cr / k^1.5 / max_{e,q} |J^-1 u|.
* Divergence and continuity penalty step, Eq. (penalty_step), after the viscous
  step: (v, u~) + (div v, tau_div div u~) + (v.n, tau_cont [u~].n) = (v, u^{n+1}).
  READING ("chosen according to Fehn2018b", formulas not printed):
  tau_div,e = ubar_e h_e/(k+1) dt, tau_cont,e = ubar_e dt (factors 1), ubar_e the
  cell mean of |u^{n+1}|, h_e = |Omega_e|^(1/3); tau_cont averaged over the two
  cells of an interior face; the jump of the normal component only; on Dirichlet
  walls the exterior state is the wall data g (the paper: the oriented jump
  incorporates the boundary data).

Cells are affine (oracle.mesh / oracle.sipg: the box, the channel) or trilinear
(oracle.mapped: the jittered channel); every form reads its geometry through
``cell_geo`` / ``face_geo`` - quadrature weights w det J, physical basis
gradients J^-T grad_xi phi, J^-1 and the outward unit normal per point - which
are constant per cell on affine grids. The element-local L2 projection onto
Q_k and the mass matrix then carry det J per point, so the same code is the
form of Sec. 5 on general hexahedra.

The oracle solves every linear system exactly (sparse LU; the pressure with a
rank-one term that fixes the mean). Pins: tests/test_oracle_splitting.py,
tests/test_oracle_channel.py.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mass as omass
from . import nonlinear
from . import viscosity
from .mapped import MappedMesh, MappedSIPG
from .mesh import BoxMesh
from .sipg import SIPG, _sym

BDF = {1: (1.0, (1.0,), (1.0,)), 2: (1.5, (2.0, -0.5), (2.0, -1.0))}
EXTRAP = {0: (), 1: (1.0,), 2: (2.0, -1.0)}


def face_normal(f):
    d, s = divmod(f, 2)
    n = np.zeros(3)
    n[d] = 2.0 * s - 1.0
    return d, s, n


def cell_geo(S, e):
    """Gauss-point weights w det J (P,), physical basis gradients (P, n^3, 3) and
    J^-1 (P, 3, 3) of cell e (per point on trilinear cells)."""
    if hasattr(S, 'cell_geometry'):
        _, J, W, Jinv = S.cell_geometry(e)
        return W, S._grad(S.cell_dphi, J), Jinv
    P = len(S.cell_w)
    return (S.cell_w * S.mesh.volume(), S._phys_grad(S.cell_dphi),
            np.broadcast_to(np.diag(1.0 / np.asarray(S.mesh.h)), (P, 3, 3)))


def face_geo(S, e, f):
    """Surface weights (P,), outward unit normals (P, 3) and physical basis gradients
    (P, n^3, 3) of cell e at the Gauss points of its face f."""
    if hasattr(S, 'face_geometry'):
        _, J, nvec, Wf = S.face_geometry(e, f)
        return Wf, nvec, S._grad(S.face_dphi[f], J)
    d, s, n = face_normal(f)
    P = len(S.face_w2)
    return S.face_w2 * S.mesh.face_area(d), np.broadcast_to(n, (P, 3)), S._phys_grad(S.face_dphi[f])


def _cell(S, x, e):
    return np.asarray(x).reshape(S.mesh.n_cells, S.ncomp, S.n ** 3)[e]


def _values(phi, U):
    """values (P, ncomp) of nodal coefficients U (ncomp, n^3) at points with basis phi (P, n^3)."""
    return np.einsum('pi,ci->pc', phi, U)


def _grads(gphys, U):
    """gradients G[p, c, l] = d u_c / d x_l from the physical basis gradients (P, n^3, 3)."""
    return np.einsum('pil,ci->pcl', gphys, U)


def wall_data(S, g_faces, e, f):
    """Dirichlet datum g at the face points of (e, f): per boundary id (the box sides 0..5,
    faces against removed cells 6; a missing id is no-slip) a constant vector or a callable
    of the points (the inflow profile, the consistency pins)."""
    b = S.mesh.boundary_id(e, f)
    g = g_faces[b] if g_faces is not None and b < len(g_faces) else np.zeros(3)
    if callable(g):
        return np.asarray(g(S.face_points(e, f)), dtype=np.float64)
    return np.broadcast_to(np.asarray(g, dtype=np.float64), (S.nq ** 2, 3))


def _exterior(S, x, e, f, g_faces):
    """Trace values and gradients of the exterior state at the face points of (e, f)."""
    mesh = S.mesh
    d, s = divmod(f, 2)
    U = _cell(S, x, e)
    um, Gm = _values(S.face_phi[f], U), _grads(face_geo(S, e, f)[2], U)
    bt = mesh.boundary_type(e, f)
    if bt == 'I':
        nb = mesh.neighbor(e, f)
        fo = 2 * d + (1 - s)
        Un = _cell(S, x, nb)
        return um, Gm, _values(S.face_phi[fo], Un), _grads(face_geo(S, nb, fo)[2], Un), bt
    if bt == 'D':
        g = wall_data(S, g_faces, e, f)
        return um, Gm, -um + 2.0 * g, Gm, bt
    return um, Gm, um, Gm, bt


def convective_vector(S, u, g_faces):
    """C_a = sum_e c_h(phi_a, u; u) (velocity space S, ncomp = 3)."""
    C = S.mesh.n_cells
    out = np.zeros((C, 3, S.n ** 3))
    for e in range(C):
        W, gphys, _ = cell_geo(S, e)
        U = _cell(S, u, e)
        uq, Gq = _values(S.cell_phi, U), _grads(gphys, U)
        conv = np.einsum('pl,pcl->pc', uq, Gq)
        out[e] += np.einsum('p,pi,pc->ci', W, S.cell_phi, conv)
        for f in range(6):
            Wf, nvec, _ = face_geo(S, e, f)
            um, _, up, _, bt = _exterior(S, u, e, f, g_faces)
            wn = np.einsum('pk,pk->p', 0.5 * (um + up), nvec)
            udag = 0.5 * (um + up) + 0.5 * np.sign(wn)[:, None] * (um - up)
            flux = wn[:, None] * (udag - um)
            out[e] += np.einsum('p,pi,pc->ci', Wf, S.face_phi[f], flux)
    return out.reshape(-1)


def convective_blocks(S, w, g_w):
    """Sparse matrix of u -> sum_e c_h(phi_a, u; w) for a fixed transport velocity w
    (Eq. convective_term_weak, linear in u), homogeneous wall data for u (u^+ = -u^-);
    w's exterior on walls from its own data g_w. The linearly implicit convective term
    of the viscous step (alpha_c = 1, u* = u^#)."""
    mesh = S.mesh
    C = mesh.n_cells
    m = S.n_dofs_cell
    n3 = S.n ** 3
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(n3), np.arange(n3), indexing='ij')

    def put(e_row, e_col, blk):
        for c in range(3):
            rows.append(e_row * m + c * n3 + ii.ravel())
            cols.append(e_col * m + c * n3 + jj.ravel())
            vals.append(blk.ravel())

    for e in range(C):
        W, dphi, _ = cell_geo(S, e)
        wq = _values(S.cell_phi, _cell(S, w, e))
        put(e, e, np.einsum('p,pi,pl,pjl->ij', W, S.cell_phi, wq, dphi))
        for f in range(6):
            d, s = divmod(f, 2)
            wm, _, wp, _, bt = _exterior(S, w, e, f, g_w)
            if bt == 'N':
                continue
            Wf, nvec, _ = face_geo(S, e, f)
            wn = np.einsum('pk,pk->p', 0.5 * (wm + wp), nvec)
            up_fac = 0.5 * (1.0 - np.sign(wn)) * wn      # coefficient of (u^+ - u^-)
            phi = S.face_phi[f]
            if bt == 'I':
                nb = mesh.neighbor(e, f)
                fo = 2 * d + (1 - s)
                put(e, e, -np.einsum('p,pi,pj->ij', Wf * up_fac, phi, phi))
                put(e, nb, np.einsum('p,pi,pj->ij', Wf * up_fac, phi, S.face_phi[fo]))
            else:  # Dirichlet, homogeneous: u^+ - u^- = -2 u^-
                put(e, e, -2.0 * np.einsum('p,pi,pj->ij', Wf * up_fac, phi, phi))
    N = S.n_dofs
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)).tocsr()


def convective_wall_rhs(S, w, g_w, g_u):
    """The wall-data part of c_h(., u; w) (u^+ = -u^- + 2 g_u), moved to the right-hand side."""
    mesh = S.mesh
    out = np.zeros((mesh.n_cells, 3, S.n ** 3))
    for e in range(mesh.n_cells):
        for f in range(6):
            if mesh.boundary_type(e, f) != 'D':
                continue
            Wf, nvec, _ = face_geo(S, e, f)
            wm, _, wp, _, _ = _exterior(S, w, e, f, g_w)
            wn = np.einsum('pk,pk->p', 0.5 * (wm + wp), nvec)
            up_fac = 0.5 * (1.0 - np.sign(wn)) * wn
            g = wall_data(S, g_u, e, f)
            out[e] -= np.einsum('p,pi,pc->ci', Wf * up_fac * 2.0, S.face_phi[f], g)
    return out.reshape(-1)


def convective_at_face(S, u, e, f):
    """(u.grad) u at the face points of (e, f) from the cell's own trace."""
    U = _cell(S, u, e)
    return np.einsum('pl,pcl->pc', _values(S.face_phi[f], U), _grads(face_geo(S, e, f)[2], U))


def l2_project_cell(S, e, values):
    """Element-local L2 projection onto Q_k of point values (P,) or (P, c) at the cell Gauss
    points, with the weights w det J of the cell."""
    W = cell_geo(S, e)[0]
    phi = S.cell_phi
    Ms = np.einsum('p,pi,pj->ij', W, phi, phi)
    v = values if values.ndim == 2 else values[:, None]
    rhs = np.einsum('p,pi,pc->ic', W, phi, v)
    coef = np.linalg.solve(Ms, rhs)  # (n^3, c)
    return coef.T if values.ndim == 2 else coef[:, 0]


def _curl(G):
    return np.stack([G[:, 2, 1] - G[:, 1, 2], G[:, 0, 2] - G[:, 2, 0], G[:, 1, 0] - G[:, 0, 1]], axis=1)


def viscous_boundary_terms(S, e, f, u_dd, rheology):
    """-nu n.(curl omega) + 2 n.(eps(u) grad nu) at the face points of (e, f) for the field u_dd."""
    _, nvec, gface = face_geo(S, e, f)
    U = _cell(S, u_dd, e)
    Gc = _grads(cell_geo(S, e)[1], U)
    omega = l2_project_cell(S, e, _curl(Gc))                       # (3, n^3)
    Gw = _grads(gface, omega)
    curl_omega = _curl(Gw)
    Gf = _grads(gface, U)
    pts_f = S.face_points(e, f)
    nu_f = viscosity.evaluate(rheology, pts_f, Gf)
    nu_c = viscosity.evaluate(rheology, S.cell_points(e), Gc)
    nu_coef = l2_project_cell(S, e, nu_c)                          # (n^3,)
    grad_nu = np.einsum('pil,i->pl', gface, nu_coef)
    eps = viscosity.strain_rate(Gf)
    return -nu_f * np.einsum('pk,pk->p', curl_omega, nvec) + 2.0 * np.einsum('pl,plk,pk->p', nvec, eps, grad_nu)


def ppe_boundary_datum(S, e, f, hist, order, dt, body, g_faces, rheology, g_hist=None):
    """h_p - (gamma0/dt) g_uhat.n at the face points of the Dirichlet face (e, f).

    hist: [u^n, u^{n-1}, ...] (velocity DoF vectors), body: b_h DoF vector or None,
    g_faces: the wall data at t_{n+1}; g_hist: the wall data at t_n, t_{n-1}, ... (None:
    steady data, g_faces at every time). d_t g(t_{n+1}) is the BDF-m approximation
    (gamma0 g(t_{n+1}) - sum_i alpha_i g(t_{n-i})) / dt (Sec. 3.2: g approximated by BDF-m)."""
    gamma0, alpha, beta = BDF[order]
    m_p = min(order - 1, 2)
    betabar = EXTRAP[m_p]
    nvec = face_geo(S, e, f)[1]
    P = S.nq ** 2

    def dn(v):  # normal component per point
        return np.einsum('pk,pk->p', v, nvec)

    nb = np.zeros(P)
    if body is not None:
        nb = dn(_values(S.face_phi[f], _cell(S, body, e)))
    g_new = dn(wall_data(S, g_faces, e, f))
    g_old = [dn(wall_data(S, g_faces if g_hist is None else g_hist[i], e, f)) for i in range(order)]
    dtg = (gamma0 * g_new - sum(alpha[i] * g_old[i] for i in range(order))) / dt
    conv_m = sum(beta[i] * dn(convective_at_face(S, hist[i], e, f)) for i in range(order))
    conv_mp = sum((betabar[i] * dn(convective_at_face(S, hist[i], e, f)) for i in range(m_p)), np.zeros(P))
    visc = np.zeros(P)
    if m_p > 0:
        u_dd = sum(betabar[i] * np.asarray(hist[i]) for i in range(m_p))
        visc = viscous_boundary_terms(S, e, f, u_dd, rheology)
    h_p = nb - dtg - conv_mp + visc
    g_uhat_n = dt / gamma0 * nb - dt / gamma0 * conv_m + sum(alpha[i] / gamma0 * g_old[i] for i in range(order))
    return h_p - gamma0 / dt * g_uhat_n


def ppe_rhs(Su, Sp, uhat, coef, boundary):
    """(gamma0/dt)[(grad q, uhat) - (q, {{uhat}}.n)] with the Dirichlet-face integrand replaced
    by ``boundary[(e, f)]`` (P,) values. Sp: pressure space with Su's Gauss rule."""
    mesh = Su.mesh
    C = mesh.n_cells
    out = np.zeros((C, Sp.n ** 3))
    for e in range(C):
        W = cell_geo(Su, e)[0]
        uq = _values(Su.cell_phi, _cell(Su, uhat, e))
        out[e] += coef * np.einsum('p,pil,pl->i', W, cell_geo(Sp, e)[1], uq)
        for f in range(6):
            Wf, nvec, _ = face_geo(Su, e, f)
            bt = mesh.boundary_type(e, f)
            if bt in ('I', 'N'):   # velocity Neumann (outflow): uhat^+ = uhat^-
                um, _, up, _, _ = _exterior(Su, uhat, e, f, None)
                out[e] -= coef * np.einsum('p,pi,p->i', Wf, Sp.face_phi[f],
                                           np.einsum('pk,pk->p', 0.5 * (um + up), nvec))
            elif bt == 'D':
                out[e] += np.einsum('p,pi,p->i', Wf, Sp.face_phi[f], boundary[(e, f)])
    return out.reshape(-1)


def projection_rhs(Su, Sp, p):
    """(div v, p)_e - (v, {{p}} n)_de for the velocity test functions."""
    mesh = Su.mesh
    C = mesh.n_cells
    out = np.zeros((C, 3, Su.n ** 3))
    for e in range(C):
        W, gphys, _ = cell_geo(Su, e)
        pq = Sp.cell_phi @ _cell(Sp, p, e)[0]
        out[e] += np.einsum('p,pic,p->ci', W, gphys, pq)
        for f in range(6):
            d, s = divmod(f, 2)
            Wf, nvec, _ = face_geo(Su, e, f)
            pm = Sp.face_phi[f] @ _cell(Sp, p, e)[0]
            bt = mesh.boundary_type(e, f)
            if bt == 'I':
                nb = mesh.neighbor(e, f)
                fo = 2 * d + (1 - s)
                pavg = 0.5 * (pm + Sp.face_phi[fo] @ _cell(Sp, p, nb)[0])
            elif bt == 'D':
                pavg = pm
            else:
                continue
            out[e] -= np.einsum('p,pi,p,pc->ci', Wf, Su.face_phi[f], pavg, nvec)
    return out.reshape(-1)


def viscous_dirichlet_rhs(S, nu_face, g_faces):
    """D_a = -(2 nu eps(phi_a) n, g) + (2 tau, phi_a.g + (phi_a.n)(g.n)) over Dirichlet faces."""
    mesh = S.mesh
    C = mesh.n_cells
    out = np.zeros((C, 3 * S.n ** 3))
    for e in range(C):
        for f in range(6):
            if mesh.boundary_type(e, f) != 'D':
                continue
            g = wall_data(S, g_faces, e, f)
            if not np.any(g):
                continue
            Wf, nvec, gface = face_geo(S, e, f)
            Vt, Gt = S._vector_basis(S.face_phi[f], gface)
            num = nu_face[e, f]
            tau = S._tau(e, None, num, num)
            epsn = np.einsum('pakl,pl->pak', _sym(Gt), nvec)
            gn = np.einsum('pk,pk->p', g, nvec)
            out[e] -= np.einsum('p,p,pak,pk->a', Wf, 2.0 * num, epsn, g)
            out[e] += np.einsum('p,p,pa->a', Wf, 2.0 * tau, np.einsum('pak,pk->pa', Vt, g)
                                + np.einsum('pak,pk->pa', Vt, nvec) * gn[:, None])
    return out.reshape(-1)


def cfl_dt(S, u, Cr):
    """Eq. (CFL_timestep_selection): Cr / k^1.5 / max_{e,q} |J^-1 u|."""
    vmax = 0.0
    for e in range(S.mesh.n_cells):
        Jinv = cell_geo(S, e)[2]
        uq = np.einsum('pkl,pl->pk', Jinv, _values(S.cell_phi, _cell(S, u, e)))
        vmax = max(vmax, float(np.sqrt((uq ** 2).sum(axis=1)).max()))
    return Cr / S.k ** 1.5 / vmax


def penalty_parameters(S, u, dt, zeta_div=1.0, zeta_cont=1.0):
    """tau_div,e = zeta ubar_e h_e / (k+1) dt, tau_cont,e = zeta ubar_e dt per cell, with
    ubar_e the cell mean of |u| and h_e = |Omega_e|^(1/3) (READING of "chosen according
    to Fehn2018b", Eq. penalty_step)."""
    C = S.mesh.n_cells
    tdiv, tcon = np.zeros(C), np.zeros(C)
    for e in range(C):
        W = cell_geo(S, e)[0]
        vol = float(np.sum(W))
        uq = _values(S.cell_phi, _cell(S, u, e))
        ubar = float(np.sum(W * np.linalg.norm(uq, axis=1)) / vol)
        tdiv[e] = zeta_div * ubar * vol ** (1.0 / 3.0) / (S.k + 1) * dt
        tcon[e] = zeta_cont * ubar * dt
    return tdiv, tcon


def penalty_blocks(S, tdiv, tcon):
    """Sparse matrix of the divergence and continuity penalty step, Eq. (penalty_step):
        (v, u)_e + (div v, tau_div,e div u)_e + (v.n, tau_F (u^- - u^+).n)_de
    with tau_F the mean of the two cells' tau_cont on interior faces and the cell's on a
    Dirichlet wall, where the exterior state is the wall data (its part goes to the
    right-hand side, ``penalty_wall_rhs``); nothing on Neumann walls."""
    mesh = S.mesh
    C = mesh.n_cells
    m = S.n_dofs_cell
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing='ij')

    def put(er, ec, blk):
        rows.append(er * m + ii.ravel())
        cols.append(ec * m + jj.ravel())
        vals.append(blk.ravel())

    for e in range(C):
        W, gphys, _ = cell_geo(S, e)
        V, G = S._vector_basis(S.cell_phi, gphys)
        div = np.einsum('qakk->qa', G)
        own = np.einsum('q,qak,qbk->ab', W, V, V) + tdiv[e] * np.einsum('q,qa,qb->ab', W, div, div)
        for f in range(6):
            d, s = divmod(f, 2)
            bt = mesh.boundary_type(e, f)
            if bt == 'N':
                continue
            Wf, nvec, gface = face_geo(S, e, f)
            Vt, _ = S._vector_basis(S.face_phi[f], gface)
            vn = np.einsum('qak,qk->qa', Vt, nvec)
            if bt == 'I':
                nb = mesh.neighbor(e, f)
                fo = 2 * d + (1 - s)
                tau = 0.5 * (tcon[e] + tcon[nb])
                Vn, _ = S._vector_basis(S.face_phi[fo], face_geo(S, nb, fo)[2])
                vnn = np.einsum('qak,qk->qa', Vn, nvec)
                own += tau * np.einsum('q,qa,qb->ab', Wf, vn, vn)
                put(e, nb, -tau * np.einsum('q,qa,qb->ab', Wf, vn, vnn))
            else:
                own += tcon[e] * np.einsum('q,qa,qb->ab', Wf, vn, vn)
        put(e, e, own)
    N = S.n_dofs
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)).tocsr()


def penalty_wall_rhs(S, tcon, g_faces):
    """(v.n, tau_cont,e g.n) over Dirichlet walls (the wall data of the oriented jump)."""
    mesh = S.mesh
    out = np.zeros((mesh.n_cells, 3 * S.n ** 3))
    for e in range(mesh.n_cells):
        for f in range(6):
            if mesh.boundary_type(e, f) != 'D':
                continue
            Wf, nvec, gface = face_geo(S, e, f)
            g = wall_data(S, g_faces, e, f)
            Vt, _ = S._vector_basis(S.face_phi[f], gface)
            out[e] += tcon[e] * np.einsum('q,qak,qk,q->a', Wf, Vt, nvec, np.einsum('pk,pk->p', g, nvec))
    return out.reshape(-1)


def penalty_step(S, u, dt, g_faces, zeta_div=1.0, zeta_cont=1.0):
    """The post-processed velocity of Eq. (penalty_step) (exact sparse solve)."""
    tdiv, tcon = penalty_parameters(S, u, dt, zeta_div, zeta_cont)
    K = penalty_blocks(S, tdiv, tcon)
    b = omass.apply_mass(S, u) + penalty_wall_rhs(S, tcon, g_faces)
    return spla.spsolve(K.tocsc(), b), tdiv, tcon


def pressure_solve(Sp_op, rhs):
    """The SIPG Laplacian's solution; with no pressure-Dirichlet face (all-Neumann) the
    mean-free solution for the mean-free right-hand side (Sec. 3.2)."""
    A = Sp_op.assemble().tocsc()
    m = Sp_op.mesh
    if any(m.boundary_type(e, f) == 'D' for e, f in m.boundary_faces()):
        return spla.spsolve(A, rhs)
    N = A.shape[0]
    r = rhs - rhs.mean()
    c = float(A.diagonal().mean()) / N
    one = np.ones((N, 1))
    K = (A + sp.csc_matrix(c * (one @ one.T))).tocsc()
    return spla.spsolve(K, r)


class Splitting:
    """State and one-step driver of the projection scheme."""

    def __init__(self, mesh, k, rheology, g_faces=None, body=None, viscosity_mode='linear', penalty_factor=1.0,
                 convective='explicit', ramp=None, t0=0.0):
        """g_faces: wall data per boundary id (constant vectors or callables of the points);
        ramp: optional scalar function of time, the wall data at time t being ramp(t) g_faces
        (the ramped inflow of the backward-facing-step benchmark)."""
        self.mesh, self.k = mesh, int(k)
        self.ramp = ramp
        self.t = float(t0)
        self.times = []
        self.rheology = rheology
        self.g_faces = [np.zeros(3) if g_faces is None or f >= len(g_faces) else
                        (g_faces[f] if callable(g_faces[f]) else np.asarray(g_faces[f], float)) for f in range(7)]
        space = MappedSIPG if isinstance(mesh, MappedMesh) else SIPG   # trilinear or affine cells
        self.Su = space(mesh, k, 3, penalty_factor=penalty_factor)
        self.Sp = space(mesh, k - 1, 1, penalty_factor=penalty_factor, n_quad=k + 1)   # mixed forms
        # the pressure is Neumann where the velocity is Dirichlet and vice versa (Sec. 3.2)
        pbc = tuple('N' if b == 'D' else 'D' for b in mesh.bc)
        self.pmesh = mesh.with_bc(pbc)
        self.Sp_op = space(self.pmesh, k - 1, 1, penalty_factor=penalty_factor)      # PPE operator
        self.body = None if body is None else np.asarray(body, dtype=np.float64)
        self.mode = viscosity_mode
        self.convective = convective   # 'explicit' (alpha_c = 0) or 'linear_implicit' (alpha_c = 1, u* = u#)
        self.hist = []
        self.p = None
        self.steps = 0

    def walls(self, t):
        """Wall data at time t (per boundary id)."""
        if self.ramp is None:
            return self.g_faces
        r = float(self.ramp(t))
        return [(lambda x, g=g: r * np.asarray(g(x))) if callable(g) else r * g for g in self.g_faces]

    def set_initial(self, u0, p0=None):
        self.hist = [np.array(u0, dtype=np.float64)]
        self.times = [self.t]
        self.p = np.zeros(self.Sp_op.n_dofs) if p0 is None else np.array(p0, dtype=np.float64)
        self.steps = 0

    def step(self, dt, picard=None, penalty=False):
        Su, Sp = self.Su, self.Sp
        order = min(2, len(self.hist))
        gamma0, alpha, beta = BDF[order]
        hist = self.hist
        # convective step
        rhs = sum(alpha[i] / dt * omass.apply_mass(Su, hist[i]) for i in range(order))
        if self.body is not None:
            rhs = rhs + omass.apply_mass(Su, self.body)
        t_new = self.times[0] + dt
        g_new = self.walls(t_new)
        g_hist = [self.walls(self.times[i]) for i in range(order)]
        conv = [convective_vector(Su, hist[i], g_hist[i]) for i in range(order)]
        rhs = rhs - sum(beta[i] * conv[i] for i in range(order))
        uhat = omass.apply_inverse_mass(Su, rhs, gamma0 / dt)
        # pressure step
        bnd = {}
        for e in range(self.mesh.n_cells):
            for f in range(6):
                if self.mesh.boundary_type(e, f) == 'D':
                    bnd[(e, f)] = ppe_boundary_datum(Su, e, f, hist, order, dt, self.body, g_new,
                                                     self.rheology, g_hist)
        rp = ppe_rhs(Su, Sp, uhat, gamma0 / dt, bnd)
        p = pressure_solve(self.Sp_op, rp)
        # projection step
        uhh = uhat + omass.apply_inverse_mass(Su, projection_rhs(Su, Sp, p), gamma0 / dt)
        # viscous step
        m = gamma0 / dt
        u_sharp = sum(beta[i] * hist[i] for i in range(order))
        nc, nf = Su.viscosity_at_points(self.rheology, u_sharp)
        b = omass.apply_mass(Su, uhh, m)
        if self.convective == 'linear_implicit':
            # alpha_c = 1: + c_h(v, u^{n+1}; u#) on the left, + sum_i beta_i c_h(v, u^{n-i}; u^{n-i})
            # on the right (Eq. viscous_step_weak); wall data of both terms on the right
            if picard is not None:
                raise ValueError("the linearly implicit convective step takes the linear-implicit viscosity")
            b = b + viscous_dirichlet_rhs(Su, nf, g_new) + sum(beta[i] * conv[i] for i in range(order))
            b = b + convective_wall_rhs(Su, u_sharp, g_new, g_new)
            K = Su.assemble(nc, nf, mass=m) + convective_blocks(Su, u_sharp, g_new)
            u_new = spla.spsolve(K.tocsc(), b)
            info = None
        elif picard is None:
            b = b + viscous_dirichlet_rhs(Su, nf, g_new)
            u_new = spla.spsolve(Su.assemble(nc, nf, mass=m).tocsc(), b)
            info = None
        else:
            if any(callable(g) or np.any(g) for g in g_new):
                raise ValueError("the implicit-viscosity step is built for zero wall velocity")
            info = nonlinear.viscous_step_picard(Su, self.rheology, b, u_sharp, m, **picard)
            u_new = info['u']
        if penalty:  # Alg. 1: post-process with the divergence and continuity penalty step
            u_new = penalty_step(Su, u_new, dt, g_new)[0]
        self.hist = [u_new] + hist[:1]
        self.times = [t_new] + self.times[:1]
        self.p = p
        self.steps += 1
        return {'uhat': uhat, 'p': p, 'uhathat': uhh, 'u': u_new, 'order': order, 'picard': info,
                'ppe_rhs': rp}
