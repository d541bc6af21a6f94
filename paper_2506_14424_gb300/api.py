"""Python face of libsipg: a thin wrapper over the C ABI of ``include/sipg.h``.

PyTorch supplies device memory and the stream; every step of the operator,
viscosity and solver path runs in the library's CUDA kernels. Function names
follow the C calls (``sipg_apply`` -> ``Context.apply`` and so on).
"""
import ctypes

import numpy as np
import torch

from . import _lib as L


class SipgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{L.ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(t, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")


def rheology_struct(rh):
    r = L.Rheology()
    r.law = L.LAW[rh['law']]
    keep = None
    if rh['law'] == 'constant':
        r.nu = float(rh['nu'])
    elif rh['law'] == 'sinker':
        c = np.ascontiguousarray(np.asarray(rh['centers'], dtype=np.float64).reshape(-1))
        keep = c
        r.n_spheres = len(c) // 3
        r.centers = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.radius, r.nu_max, r.nu_matrix = float(rh['radius']), float(rh['nu_max']), float(rh['nu_matrix'])
    elif rh['law'] == 'carreau':
        r.eta0, r.eta_inf, r.kappa = float(rh['eta0']), float(rh['eta_inf']), float(rh['kappa'])
        r.lam, r.a, r.b = float(rh['lam']), float(rh['a']), float(rh['b'])
    return r, keep


class Context:
    """One mesh, degree and multigrid hierarchy on the current CUDA device."""

    def __init__(self, nx, ny, nz, k_u, extent=(1.0, 1.0, 1.0), bc_velocity="DDDDDD", bc_pressure="NNNNNN",
                 penalty_factor=1.0, face_nu="max", mg_precision="f32", cheb_degree=3, cheb_range=20.0,
                 cheb_lmax_factor=1.2, lanczos_steps=15, coarse_max_dofs=2000, seed=0, krylov_arith="f64",
                 stream=None, vertices=None, mg_cph="auto", active=None, periodic=(False, False, False), mg_setup_lag=1,
                 origin=(0.0, 0.0, 0.0), bc_removed="DN"):
        """vertices: optional (nz+1, ny+1, nx+1, 3) host array of vertex positions
        (trilinear cells; fine level only, see include/sipg.h).
        active: optional (nz, ny, nx) flags of the grid cells (False = removed, e.g. the
        block below a backward-facing step); periodic: per direction; origin: lower
        corner of the grid; bc_removed: velocity and pressure condition on faces
        against removed cells (see sipg_mesh_desc).
        mg_cph: 'auto' (the cph hierarchy of Sec. 5.4 on a plain box, DG levels on any
        other mesh), True (cph; plain boxes only) or False (DG on every level)."""
        self._lib = L.load()
        m = L.MeshDesc()
        m.nx, m.ny, m.nz = int(nx), int(ny), int(nz)
        m.lx, m.ly, m.lz = (float(v) for v in extent)
        for i in range(6):
            m.bc_velocity[i] = L.BC[bc_velocity[i]]
            m.bc_pressure[i] = L.BC[bc_pressure[i]]
        act = None
        if active is not None:
            act = np.ascontiguousarray(np.asarray(active, dtype=np.uint8).reshape(-1))
            if act.size != int(nx) * int(ny) * int(nz):
                raise ValueError("active: (nz, ny, nx) flags expected")
            m.active = act.ctypes.data
        m.bc_removed_velocity = L.BC[bc_removed[0]]
        m.bc_removed_pressure = L.BC[bc_removed[1]]
        for d in range(3):
            m.periodic[d] = int(bool(periodic[d]))
            m.origin[d] = float(origin[d])
        verts = None
        if vertices is not None:
            verts = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64).reshape(-1))
            if verts.size != (int(nx) + 1) * (int(ny) + 1) * (int(nz) + 1) * 3:
                raise ValueError("vertices: (nz+1, ny+1, nx+1, 3) values expected")
            m.vertices = verts.ctypes.data
        o = L.Opts()
        o.k_u = int(k_u)
        o.penalty_factor = float(penalty_factor)
        o.face_nu = L.FACE_NU[face_nu]
        o.mg_precision = L.PREC[mg_precision]
        o.cheb_degree = int(cheb_degree)
        o.cheb_range = float(cheb_range)
        o.cheb_lmax_factor = float(cheb_lmax_factor)
        o.lanczos_steps = int(lanczos_steps)
        o.coarse_max_dofs = int(coarse_max_dofs)
        o.seed = int(seed)
        o.krylov_arith = L.PREC[krylov_arith]
        if mg_cph not in ("auto", True, False):
            raise ValueError("mg_cph: 'auto', True or False")
        o.mg_cph = L.MG_AUTO if mg_cph == "auto" else int(bool(mg_cph))
        o.mg_setup_lag = int(mg_setup_lag)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self._lib.sipg_create(ctypes.byref(m), ctypes.byref(o), ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(h))
        del verts, act  # copied by sipg_create
        if rc != L.SIPG_OK:
            raise SipgError(rc, "sipg_create failed (see stderr)")
        self._h = h
        self.k_u = int(k_u)
        self.cells = (int(nx), int(ny), int(nz))
        self.n_cells = self.n_dofs("poisson") // self.k_u ** 3

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sipg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != L.SIPG_OK:
            raise SipgError(rc, self._lib.sipg_last_error(self._h).decode())

    # ---------------------------------------------------------------- sizes
    def num_levels(self, op="viscous"):
        n = ctypes.c_int()
        self._check(self._lib.sipg_num_levels(self._h, L.OP[op], ctypes.byref(n)))
        return n.value

    def level_info(self, op="viscous", level=0):
        cells = (ctypes.c_int * 3)()
        k = ctypes.c_int()
        nd = ctypes.c_int64()
        self._check(self._lib.sipg_level_info(self._h, L.OP[op], level, ctypes.byref(cells), ctypes.byref(k),
                                              ctypes.byref(nd)))
        return tuple(cells), k.value, nd.value

    def n_dofs(self, op="viscous", level=0):
        return self.level_info(op, level)[2]

    # ------------------------------------------------------------ viscosity
    def set_viscosity(self, rheology, u_lin=None):
        r, keep = rheology_struct(rheology)
        if u_lin is not None:
            _need_cuda(u_lin, torch.float64)
        self._check(self._lib.sipg_set_viscosity(self._h, ctypes.byref(r), _ptr(u_lin)))
        del keep

    def get_viscosity(self, level=0):
        _, k, _ = self.level_info("viscous", level)
        n = k + 1
        C = self.level_cells("viscous", level)
        dev = torch.device("cuda")
        nc = torch.empty(C * n ** 3, dtype=torch.float64, device=dev)
        nf = torch.empty(C * 6 * n * n, dtype=torch.float64, device=dev)
        self._check(self._lib.sipg_get_viscosity(self._h, level, _ptr(nc), _ptr(nf)))
        return nc.view(C, n ** 3), nf.view(C, 6, n * n)

    # ---------------------------------------------------------------- apply
    def apply(self, op, x, y=None, mass=0.0, level=0, arith=None):
        """y = (mass M + A) x; arith 'f64' (default for double), 'f64ff' or 'f32'."""
        _need_cuda(x)
        prec = L.PREC[arith or ("f64" if x.dtype == torch.float64 else "f32")]
        if (prec == L.PREC["f32"]) != (x.dtype == torch.float32):
            raise TypeError("f32 arithmetic needs float32 vectors, f64/f64ff need float64")
        if y is None:
            y = torch.empty_like(x)
        _need_cuda(y, x.dtype)
        if x.numel() != self.n_dofs(op, level) or y.numel() != x.numel():
            raise ValueError("vector size does not match the level")
        self._check(self._lib.sipg_level_apply(self._h, L.OP[op], level, prec, _ptr(x), _ptr(y), float(mass)))
        return y

    def mass(self, op, x, y=None, coeff=1.0, arith=None, inverse=False):
        """y = coeff M x (or (coeff M)^-1 x with inverse=True), cell mass matrix of op."""
        _need_cuda(x)
        prec = L.PREC[arith or ("f64" if x.dtype == torch.float64 else "f32")]
        if (prec == L.PREC["f32"]) != (x.dtype == torch.float32):
            raise TypeError("f32 arithmetic needs float32 vectors, f64/f64ff need float64")
        if y is None:
            y = torch.empty_like(x)
        _need_cuda(y, x.dtype)
        if x.numel() != self.n_dofs(op) or y.numel() != x.numel():
            raise ValueError("vector size does not match the fine level")
        fn = self._lib.sipg_inverse_mass_apply if inverse else self._lib.sipg_mass_apply
        self._check(fn(self._h, L.OP[op], prec, _ptr(x), _ptr(y), float(coeff)))
        return y

    def ff_convert(self, x):
        """Float-float split (hi, lo) and its binary64 recombination, as the kernels do it."""
        _need_cuda(x, torch.float64)
        hilo = torch.empty(2 * x.numel(), dtype=torch.float32, device=x.device)
        back = torch.empty_like(x)
        self._check(self._lib.sipg_ff_convert(self._h, _ptr(x), _ptr(hilo), _ptr(back), x.numel()))
        return hilo.view(-1, 2), back

    def picard_solve(self, rheology, b, u, mass=0.0, rtol=1e-6, atol=1e-12, maxit=20, aitken=True,
                     omega_init=1.0, lin_rtol=1e-3, lin_atol=0.0, lin_maxit=500, precond="mg", check=True):
        """Nonlinear viscous step by Picard/Aitken; u: initial guess in, last iterate out."""
        _need_cuda(b, torch.float64)
        _need_cuda(u, torch.float64)
        r, keep = rheology_struct(rheology)
        o = L.PicardOpts()
        self._lib.sipg_default_picard_opts(ctypes.byref(o))
        o.mass_coeff, o.rtol, o.atol, o.maxit = float(mass), float(rtol), float(atol), int(maxit)
        o.aitken, o.omega_init = int(bool(aitken)), float(omega_init)
        o.lin_rtol, o.lin_atol, o.lin_maxit = float(lin_rtol), float(lin_atol), int(lin_maxit)
        o.precond = L.PRECOND[precond]
        cap = int(maxit) + 1
        res_h = (ctypes.c_double * cap)()
        om_h = (ctypes.c_double * cap)()
        st = L.PicardStats()
        st.history_len = cap
        st.residuals = ctypes.cast(res_h, ctypes.POINTER(ctypes.c_double))
        st.omegas = ctypes.cast(om_h, ctypes.POINTER(ctypes.c_double))
        rc = self._lib.sipg_picard_solve(self._h, ctypes.byref(r), _ptr(b), _ptr(u), ctypes.byref(o),
                                         ctypes.byref(st))
        del keep
        if check and rc not in (L.SIPG_OK, -4):
            self._check(rc)
        k = st.iterations
        return {"status": rc, "iterations": k, "lin_iterations": st.lin_iterations, "res0": st.res0,
                "res": st.res, "seconds": st.seconds, "residuals": list(res_h[:k + 1]), "omegas": list(om_h[:k])}

    # ------------------------------------------------ splitting step
    @staticmethod
    def _wall(wall):
        if wall is None:
            return None
        w = np.ascontiguousarray(np.asarray(wall, dtype=np.float64).reshape(18))
        return w

    def convective(self, u, wall=None, y=None):
        """y = C(u) = c_h(., u; u) with wall velocity wall (6 x 3, box sides -x..+z)."""
        _need_cuda(u, torch.float64)
        y = torch.empty_like(u) if y is None else y
        w = self._wall(wall)
        wp = w.ctypes.data_as(ctypes.c_void_p) if w is not None else None
        self._check(self._lib.sipg_convective_apply(self._h, wp, _ptr(u), _ptr(y)))
        return y

    def convective_lin(self, w, u, wall_w=None, wall_u=None):
        """y = sum_e c_h(., u; w) (linear in u; see sipg_convective_lin_apply)."""
        _need_cuda(w, torch.float64)
        _need_cuda(u, torch.float64)
        y = torch.empty_like(u)
        ww, wu = self._wall(wall_w), self._wall(wall_u)
        self._check(self._lib.sipg_convective_lin_apply(
            self._h, _ptr(w), ww.ctypes.data_as(ctypes.c_void_p) if ww is not None else None,
            wu.ctypes.data_as(ctypes.c_void_p) if wu is not None else None, _ptr(u), _ptr(y)))
        return y

    def projection_rhs(self, p):
        _need_cuda(p, torch.float64)
        y = torch.empty(self.n_dofs("viscous"), dtype=torch.float64, device=p.device)
        self._check(self._lib.sipg_projection_rhs(self._h, _ptr(p), _ptr(y)))
        return y

    def viscous_wall_rhs(self, wall):
        y = torch.empty(self.n_dofs("viscous"), dtype=torch.float64, device="cuda")
        w = self._wall(wall)
        self._check(self._lib.sipg_viscous_wall_rhs(self._h, w.ctypes.data_as(ctypes.c_void_p), _ptr(y)))
        return y

    def cfl_dt(self, u, courant):
        _need_cuda(u, torch.float64)
        dt = ctypes.c_double()
        self._check(self._lib.sipg_cfl_dt(self._h, _ptr(u), float(courant), ctypes.byref(dt)))
        return dt.value

    def penalty_tau(self, u, dt, zeta_div=1.0, zeta_cont=1.0):
        """(tau_div, tau_cont) per cell of the penalty step (see sipg_penalty_tau)."""
        _need_cuda(u, torch.float64)
        nc = self.n_cells
        td = torch.empty(nc, dtype=torch.float64, device=u.device)
        tc = torch.empty(nc, dtype=torch.float64, device=u.device)
        self._check(self._lib.sipg_penalty_tau(self._h, _ptr(u), float(dt), float(zeta_div), float(zeta_cont),
                                               _ptr(td), _ptr(tc)))
        return td, tc

    def penalty_apply(self, tau_div, tau_cont, x):
        """y = K x, the penalty step's operator (see sipg_penalty_apply)."""
        for t in (tau_div, tau_cont, x):
            _need_cuda(t, torch.float64)
        y = torch.empty_like(x)
        self._check(self._lib.sipg_penalty_apply(self._h, _ptr(tau_div), _ptr(tau_cont), _ptr(x), _ptr(y)))
        return y

    def penalty_wall_rhs(self, wall, tau_cont):
        _need_cuda(tau_cont, torch.float64)
        y = torch.empty(self.n_dofs("viscous"), dtype=torch.float64, device=tau_cont.device)
        w = self._wall(wall)
        wp = w.ctypes.data_as(ctypes.c_void_p) if w is not None else None
        self._check(self._lib.sipg_penalty_wall_rhs(self._h, wp, _ptr(tau_cont), _ptr(y)))
        return y

    def penalty_step(self, u, dt, wall=None, zeta_div=1.0, zeta_cont=1.0, rtol=1e-10, maxit=500, out=None):
        """The divergence and continuity penalty step of Eq. (penalty_step) (see sipg_penalty_step)."""
        _need_cuda(u, torch.float64)
        out = torch.empty_like(u) if out is None else out
        w = self._wall(wall)
        wp = w.ctypes.data_as(ctypes.c_void_p) if w is not None else None
        its, res = ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.sipg_penalty_step(self._h, wp, _ptr(u), float(dt), float(zeta_div), float(zeta_cont),
                                                float(rtol), int(maxit), _ptr(out), ctypes.byref(its),
                                                ctypes.byref(res)))
        return out, {"iterations": its.value, "rel_residual": res.value}

    def rhs_manufactured(self, case="velocity"):
        """Load vector of a manufactured solution (see sipg_rhs_manufactured)."""
        op = "viscous" if case == "velocity" else "poisson"
        b = torch.empty(self.n_dofs(op), dtype=torch.float64, device="cuda")
        self._check(self._lib.sipg_rhs_manufactured(self._h, 0 if case == "velocity" else 1, _ptr(b)))
        return b

    def boundary_faces(self):
        """(cell, face, boundary id) of every boundary face of the velocity mesh, (nbf, 3) ints,
        in the order of the step's wall_points arrays."""
        nbf = ctypes.c_int()
        self._check(self._lib.sipg_boundary_faces(self._h, ctypes.byref(nbf), None, None))
        out = np.zeros((nbf.value, 3), dtype=np.int32)
        self._check(self._lib.sipg_boundary_faces(self._h, ctypes.byref(nbf),
                                                  out.ctypes.data_as(ctypes.c_void_p), None))
        return out

    def boundary_points(self):
        """Positions of the Gauss points of every boundary face, (nbf, n^2, 3) on the device."""
        nbf = ctypes.c_int()
        self._check(self._lib.sipg_boundary_faces(self._h, ctypes.byref(nbf), None, None))
        n = self.k_u + 1
        out = torch.empty((nbf.value, n * n, 3), dtype=torch.float64, device="cuda")
        self._check(self._lib.sipg_boundary_faces(self._h, ctypes.byref(nbf), None, _ptr(out)))
        return out

    def step_init(self, u0, p0=None):
        _need_cuda(u0, torch.float64)
        self._check(self._lib.sipg_step_init(self._h, _ptr(u0), _ptr(p0)))

    def solve_convective(self, w, b, x=None, wall=None, rtol=1e-8, atol=0.0, maxit=500, precond="mg", mass=0.0,
                         restart=30, check=True):
        """GMRES solve of ((mass M + A(nu)) + C(w)) x = b (see sipg_solve_convective)."""
        _need_cuda(b, torch.float64)
        if w is not None:
            _need_cuda(w, torch.float64)
        x = torch.zeros_like(b) if x is None else x
        so = L.SolveOpts(float(rtol), float(atol), int(maxit), L.PRECOND[precond], float(mass))
        st = L.SolveStats()
        wl = self._wall(wall)
        wp = wl.ctypes.data_as(ctypes.c_void_p) if wl is not None else None
        rc = self._lib.sipg_solve_convective(self._h, _ptr(w), wp, _ptr(b), _ptr(x), ctypes.byref(so), int(restart),
                                             ctypes.byref(st))
        if check:
            self._check(rc)
        return x, {"iterations": st.iterations, "rel_residual": st.rel_residual, "seconds": st.seconds,
                   "status": rc}

    def step(self, rheology, dt, wall=None, body=None, viscosity_mode="linear", ppe_rtol=1e-8, visc_rtol=1e-8,
             maxit=1000, picard=None, convective_mode="explicit", gmres_restart=30, penalty=False,
             penalty_rtol=1e-10, wall_points=None, wall_points_prev=None):
        """One step of the projection scheme (see include/sipg.h, sipg_step)."""
        r, keep = rheology_struct(rheology)
        o = L.StepOpts()
        self._lib.sipg_default_step_opts(ctypes.byref(o))
        o.dt = float(dt)
        if wall is not None:
            for i, v in enumerate(np.asarray(wall, dtype=np.float64).reshape(18)):
                o.wall_velocity[i] = float(v)
        if body is not None:
            _need_cuda(body, torch.float64)
            o.body = body.data_ptr()
        o.viscosity_mode = L.VISC_MODE[viscosity_mode]
        o.convective_mode = L.CONV_MODE[convective_mode]
        o.gmres_restart = int(gmres_restart)
        o.ppe_rtol, o.visc_rtol, o.maxit = float(ppe_rtol), float(visc_rtol), int(maxit)
        o.penalty, o.penalty_rtol = int(bool(penalty)), float(penalty_rtol)
        for name, wp in (("wall_points", wall_points), ("wall_points_prev", wall_points_prev)):
            if wp is not None:
                _need_cuda(wp, torch.float64)
                setattr(o, name, wp.data_ptr())
        for key, val in (picard or {}).items():
            setattr(o.picard, key, val)
        st = L.StepStats()
        self._check(self._lib.sipg_step(self._h, ctypes.byref(r), ctypes.byref(o), ctypes.byref(st)))
        del keep
        return {f: getattr(st, f) for f, _ in L.StepStats._fields_}

    def step_field(self, which):
        n = self.n_dofs("poisson") if which in ("p", "ppe_rhs") else self.n_dofs("viscous")
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        self._check(self._lib.sipg_step_field(self._h, L.FIELD[which], _ptr(out)))
        return out

    def apply_host(self, op, x, mass=0.0, out=None):
        """y = (mass M + A) x for host arrays (copies inside the call). Pinned host
        memory (e.g. numpy views of torch.empty(..., pin_memory=True)) copies at
        the link's speed; out: optional preallocated result array."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.size != self.n_dofs(op):
            raise ValueError("vector size does not match the fine level")
        if out is None:
            y = np.empty_like(x)
        else:
            y = out
            if not (isinstance(y, np.ndarray) and y.dtype == np.float64 and y.flags.c_contiguous and y.size == x.size):
                raise ValueError("out: contiguous float64 array of the vector's size")
        self._check(self._lib.sipg_apply_host(self._h, L.OP[op], x.ctypes.data_as(ctypes.c_void_p),
                                              y.ctypes.data_as(ctypes.c_void_p), float(mass)))
        return y

    def apply_host_static(self, op, x, mass=0.0):
        """apply_host without device allocation: fixed 524,288-value staging
        area shared by all calls on the device (see include/sipg.h)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.size != self.n_dofs(op):
            raise ValueError("vector size does not match the fine level")
        y = np.empty_like(x)
        self._check(self._lib.sipg_apply_host_static(self._h, L.OP[op], x.ctypes.data_as(ctypes.c_void_p),
                                                     y.ctypes.data_as(ctypes.c_void_p), float(mass)))
        return y

    # ---------------------------------------------------------------- solve
    def solve(self, op, b, x=None, rtol=1e-8, atol=0.0, maxit=500, precond="mg", mass=0.0, check=True):
        _need_cuda(b, torch.float64)
        if x is None:
            x = torch.zeros_like(b)
        _need_cuda(x, torch.float64)
        so = L.SolveOpts(float(rtol), float(atol), int(maxit), L.PRECOND[precond], float(mass))
        st = L.SolveStats()
        rc = self._lib.sipg_solve(self._h, L.OP[op], _ptr(b), _ptr(x), ctypes.byref(so), ctypes.byref(st))
        stats = {"iterations": st.iterations, "rel_residual": st.rel_residual, "seconds": st.seconds,
                 "status": st.status}
        if check and rc != L.SIPG_OK:
            raise SipgError(rc, self._lib.sipg_last_error(self._h).decode())
        return x, stats

    # ------------------------------------------------------- multigrid bits
    def inverse_diagonal(self, op="viscous", level=0):
        out = torch.empty(self.n_dofs(op, level), dtype=torch.float64, device="cuda")
        self._check(self._lib.sipg_get_inverse_diagonal(self._h, L.OP[op], level, _ptr(out)))
        return out

    def lmax_estimate(self, op="viscous", level=0):
        v = ctypes.c_double()
        self._check(self._lib.sipg_get_lmax_estimate(self._h, L.OP[op], level, ctypes.byref(v)))
        return v.value

    def transfer(self, op, level, direction, x):
        _need_cuda(x)
        prec = L.PREC["f64" if x.dtype == torch.float64 else "f32"]
        n_out = self.n_dofs(op, level if direction > 0 else level + 1)
        out = torch.empty(n_out, dtype=x.dtype, device=x.device)
        self._check(self._lib.sipg_transfer(self._h, L.OP[op], level, int(direction), prec, _ptr(x), _ptr(out)))
        return out

    def smooth(self, op, level, b, x):
        _need_cuda(b)
        _need_cuda(x, b.dtype)
        prec = L.PREC["f64" if b.dtype == torch.float64 else "f32"]
        self._check(self._lib.sipg_smooth(self._h, L.OP[op], level, prec, _ptr(b), _ptr(x)))
        return x

    def vcycle(self, op, b):
        _need_cuda(b, torch.float64)
        x = torch.empty_like(b)
        self._check(self._lib.sipg_vcycle(self._h, L.OP[op], _ptr(b), _ptr(x)))
        return x

    def level_cells(self, op="viscous", level=0):
        """Active cells of a level (the grid's cells on a plain box)."""
        _, k, nd = self.level_info(op, level)
        return nd // ((3 if op == "viscous" else 1) * (k + 1) ** 3)

    def node_points(self, op="viscous", level=0):
        _, k, _ = self.level_info(op, level)
        n = k + 1
        out = np.empty((self.level_cells(op, level), n ** 3, 3))
        self._check(self._lib.sipg_node_points(self._h, L.OP[op], level, out.ctypes.data_as(ctypes.c_void_p)))
        return out


class Server:
    """Continuous-batching solve server (see include/sipg.h, sipg_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots=8, mg_precision="f32", cheb_degree=3, krylov_arith="f64"):
        self._lib = L.load()
        o = L.ServerOpts(int(hbm_budget_bytes), int(max_slots), L.PREC[mg_precision], int(cheb_degree),
                         L.PREC[krylov_arith])
        h = ctypes.c_void_p()
        rc = self._lib.sipg_server_create(ctypes.byref(o), ctypes.byref(h))
        if rc != L.SIPG_OK:
            raise SipgError(rc, "sipg_server_create failed")
        self._h = h
        self._sizes = {}

    def submit(self, n_cells, k_u, rheology, rtol=1e-8, maxit=300, seed=0, keep_solution=False,
               rhs="manufactured"):
        """Queue a viscous solve on the n^3 unit cube. rheology: a constant, analytic or
        sinker dict; rhs: "manufactured" (b = A u*, u* from seed), "buoyancy" (b = M f of the
        spheres), a host numpy array (copied now) or a CUDA torch tensor (read at admission:
        keep it alive and unchanged until the request is done)."""
        r_struct, keep = rheology_struct(rheology)
        b_ptr = None
        if isinstance(rhs, str):
            kind = L.RHS[rhs]
        elif isinstance(rhs, np.ndarray):
            kind = L.RHS["host"]
            b_host = np.ascontiguousarray(rhs, dtype=np.float64)
            b_ptr = b_host.ctypes.data
        else:  # a device tensor
            kind = L.RHS["device"]
            assert rhs.is_cuda and rhs.dtype == torch.float64 and rhs.is_contiguous()
            b_ptr = rhs.data_ptr()
        r = L.Request(int(n_cells), int(k_u), ctypes.pointer(r_struct), kind, b_ptr, float(rtol), int(maxit),
                      int(seed), int(bool(keep_solution)))
        rid = ctypes.c_uint64()
        rc = self._lib.sipg_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid))
        del keep
        if rc != L.SIPG_OK:
            raise SipgError(rc, "sipg_server_submit failed")
        self._sizes[rid.value] = (int(n_cells) ** 3 * 3 * (int(k_u) + 1) ** 3, bool(keep_solution))
        return rid.value

    def poll(self, rid):
        """None while pending, else (result dict, solution or None)."""
        res = L.Result()
        n, keep = self._sizes.get(rid, (0, False))
        x = np.empty(n) if keep else None
        rc = self._lib.sipg_server_poll(self._h, ctypes.c_uint64(rid), ctypes.byref(res),
                                        x.ctypes.data_as(ctypes.c_void_p) if keep else None)
        if rc == L.SIPG_PENDING:
            return None
        if rc != L.SIPG_OK:
            raise SipgError(rc, "sipg_server_poll failed")
        out = {f: getattr(res, f) for f, _ in L.Result._fields_}
        return out, x

    def drain(self, timeout=0.0):
        rc = self._lib.sipg_server_drain(self._h, float(timeout))
        if rc != L.SIPG_OK:
            raise SipgError(rc, self._lib.sipg_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sipg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alu_peak(prec):
    """FMA throughput of the current device in TFLOP/s: prec "f64" or "f32" (sipg_alu_peak)."""
    lib = L.load()
    t = ctypes.c_double()
    rc = lib.sipg_alu_peak(L.PREC[prec], ctypes.byref(t))
    if rc != L.SIPG_OK:
        raise SipgError(rc, "sipg_alu_peak failed")
    return t.value


def estimate_bytes(n_cells, k_u):
    """Device bytes of a context for an n^3 unit-cube mesh of degree k_u."""
    lib = L.load()
    m = L.MeshDesc()
    m.nx = m.ny = m.nz = int(n_cells)
    m.lx = m.ly = m.lz = 1.0
    for i in range(6):
        m.bc_velocity[i] = 0
        m.bc_pressure[i] = 1
    o = L.Opts()
    lib.sipg_default_opts(ctypes.byref(o))
    o.k_u = int(k_u)
    b = ctypes.c_int64()
    rc = lib.sipg_estimate_bytes(ctypes.byref(m), ctypes.byref(o), ctypes.byref(b))
    if rc != L.SIPG_OK:
        raise SipgError(rc, "sipg_estimate_bytes failed")
    return b.value
