"""ctypes binding of libsipg (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python
arguments to the C structs of ``include/sipg.h`` and passes device pointers of
caller-owned torch tensors through. It never falls back to a CPU path: if the
shared library is missing or fails to load, it raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsipg.so")

SIPG_OK, SIPG_PENDING = 0, 1
ERRORS = {-1: "SIPG_ERR_INVALID", -2: "SIPG_ERR_CUDA", -3: "SIPG_ERR_NOMEM", -4: "SIPG_ERR_MAXIT",
          -5: "SIPG_ERR_BREAKDOWN", -6: "SIPG_ERR_NAN", -7: "SIPG_ERR_TIMEOUT", -8: "SIPG_ERR_STATE"}
OP = {"viscous": 0, "poisson": 1}
PREC = {"f64": 0, "f32": 1, "f64ff": 2}
LAW = {"constant": 0, "analytic": 1, "sinker": 2, "carreau": 3}
PRECOND = {"none": 0, "jacobi": 1, "mg": 2}
MG_AUTO, MG_DG, MG_CPH = -1, 0, 1
FACE_NU = {"max": 0, "arith": 1, "harmonic": 2}
BC = {"D": 0, "N": 1}

# Every symbol declared in include/sipg.h (checked by the CPU test suite).
EXPORTS = [
    "sipg_default_opts", "sipg_create", "sipg_destroy", "sipg_last_error", "sipg_num_levels",
    "sipg_level_info", "sipg_set_viscosity", "sipg_apply", "sipg_apply_host", "sipg_level_apply",
    "sipg_solve", "sipg_get_viscosity", "sipg_get_inverse_diagonal", "sipg_get_lmax_estimate",
    "sipg_transfer", "sipg_smooth", "sipg_vcycle", "sipg_node_points", "sipg_apply_host_static",
    "sipg_estimate_bytes", "sipg_server_create", "sipg_server_submit", "sipg_server_poll", "sipg_server_drain",
    "sipg_server_last_error", "sipg_server_destroy", "sipg_mass_apply", "sipg_inverse_mass_apply",
    "sipg_default_picard_opts", "sipg_picard_solve", "sipg_ff_convert", "sipg_default_step_opts",
    "sipg_step_init", "sipg_step", "sipg_step_field", "sipg_cfl_dt", "sipg_convective_apply",
    "sipg_projection_rhs", "sipg_viscous_wall_rhs", "sipg_solve_convective", "sipg_convective_lin_apply",
    "sipg_penalty_tau", "sipg_penalty_apply", "sipg_penalty_wall_rhs", "sipg_penalty_step",
    "sipg_boundary_faces", "sipg_rhs_manufactured", "sipg_topology_tables", "sipg_coarsen_mask",
    "sipg_level_plan", "sipg_alu_peak",
]
FIELD = {"u": 0, "p": 1, "uhat": 2, "uhathat": 3, "ppe_rhs": 4, "u_prev": 5}
VISC_MODE = {"linear": 0, "implicit": 1}
CONV_MODE = {"explicit": 0, "linear_implicit": 1}


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("bc_velocity", ctypes.c_int * 6), ("bc_pressure", ctypes.c_int * 6),
                ("vertices", ctypes.c_void_p), ("active", ctypes.c_void_p),
                ("bc_removed_velocity", ctypes.c_int), ("bc_removed_pressure", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("origin", ctypes.c_double * 3)]


class Opts(ctypes.Structure):
    _fields_ = [("k_u", ctypes.c_int), ("penalty_factor", ctypes.c_double), ("face_nu", ctypes.c_int),
                ("mg_precision", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("cheb_range", ctypes.c_double),
                ("cheb_lmax_factor", ctypes.c_double), ("lanczos_steps", ctypes.c_int),
                ("coarse_max_dofs", ctypes.c_int), ("seed", ctypes.c_uint64), ("krylov_arith", ctypes.c_int),
                ("mg_cph", ctypes.c_int), ("mg_setup_lag", ctypes.c_int)]


class Rheology(ctypes.Structure):
    _fields_ = [("law", ctypes.c_int), ("nu", ctypes.c_double), ("n_spheres", ctypes.c_int),
                ("centers", ctypes.POINTER(ctypes.c_double)), ("radius", ctypes.c_double),
                ("nu_max", ctypes.c_double), ("nu_matrix", ctypes.c_double), ("eta0", ctypes.c_double),
                ("eta_inf", ctypes.c_double), ("kappa", ctypes.c_double), ("lam", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("precond", ctypes.c_int), ("mass_coeff", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]


class PicardOpts(ctypes.Structure):
    _fields_ = [("mass_coeff", ctypes.c_double), ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("aitken", ctypes.c_int), ("omega_init", ctypes.c_double),
                ("lin_rtol", ctypes.c_double), ("lin_atol", ctypes.c_double), ("lin_maxit", ctypes.c_int),
                ("precond", ctypes.c_int)]


class PicardStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("lin_iterations", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("history_len", ctypes.c_int), ("residuals", ctypes.POINTER(ctypes.c_double)),
                ("omegas", ctypes.POINTER(ctypes.c_double))]


class StepOpts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("wall_velocity", ctypes.c_double * 18),
                ("body", ctypes.c_void_p), ("viscosity_mode", ctypes.c_int), ("convective_mode", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("ppe_rtol", ctypes.c_double),
                ("visc_rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("picard", PicardOpts),
                ("penalty", ctypes.c_int), ("penalty_rtol", ctypes.c_double),
                ("wall_points", ctypes.c_void_p), ("wall_points_prev", ctypes.c_void_p)]


class StepStats(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("ppe_iterations", ctypes.c_int), ("visc_iterations", ctypes.c_int),
                ("picard_updates", ctypes.c_int), ("ppe_rel_residual", ctypes.c_double),
                ("visc_rel_residual", ctypes.c_double), ("t_convective", ctypes.c_double),
                ("t_pressure", ctypes.c_double), ("t_projection", ctypes.c_double),
                ("t_viscous", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("penalty_iterations", ctypes.c_int), ("t_penalty", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int), ("mg_precision", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("krylov_arith", ctypes.c_int)]


RHS = {"manufactured": 0, "buoyancy": 1, "host": 2, "device": 3}


class Request(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("k_u", ctypes.c_int), ("rheology", ctypes.POINTER(Rheology)),
                ("rhs", ctypes.c_int), ("b", ctypes.c_void_p), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("seed", ctypes.c_uint64), ("keep_solution", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("err_vs_ustar", ctypes.c_double), ("n_dofs", ctypes.c_int64), ("queue_s", ctypes.c_double),
                ("solve_s", ctypes.c_double), ("latency_s", ctypes.c_double)]


_lib = None


def load(path=None):
    """Load libsipg.so (raises OSError/RuntimeError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsipg is not built ({p} missing): run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "sipg_default_opts": (None, [P(Opts)]),
        "sipg_create": (i, [P(MeshDesc), P(Opts), vp, P(vp)]),
        "sipg_destroy": (i, [vp]),
        "sipg_last_error": (ctypes.c_char_p, [vp]),
        "sipg_num_levels": (i, [vp, i, P(i)]),
        "sipg_level_info": (i, [vp, i, i, P(ctypes.c_int * 3), P(i), P(i64)]),
        "sipg_set_viscosity": (i, [vp, P(Rheology), vp]),
        "sipg_apply": (i, [vp, i, i, vp, vp, d]),
        "sipg_apply_host": (i, [vp, i, vp, vp, d]),
        "sipg_apply_host_static": (i, [vp, i, vp, vp, d]),
        "sipg_level_apply": (i, [vp, i, i, i, vp, vp, d]),
        "sipg_solve": (i, [vp, i, vp, vp, P(SolveOpts), P(SolveStats)]),
        "sipg_get_viscosity": (i, [vp, i, vp, vp]),
        "sipg_get_inverse_diagonal": (i, [vp, i, i, vp]),
        "sipg_get_lmax_estimate": (i, [vp, i, i, P(d)]),
        "sipg_transfer": (i, [vp, i, i, i, i, vp, vp]),
        "sipg_smooth": (i, [vp, i, i, i, vp, vp]),
        "sipg_vcycle": (i, [vp, i, vp, vp]),
        "sipg_node_points": (i, [vp, i, i, vp]),
        "sipg_estimate_bytes": (i, [P(MeshDesc), P(Opts), P(i64)]),
        "sipg_server_create": (i, [P(ServerOpts), P(vp)]),
        "sipg_server_submit": (i, [vp, P(Request), P(ctypes.c_uint64)]),
        "sipg_server_poll": (i, [vp, ctypes.c_uint64, P(Result), vp]),
        "sipg_server_drain": (i, [vp, d]),
        "sipg_server_last_error": (ctypes.c_char_p, [vp]),
        "sipg_server_destroy": (i, [vp]),
        "sipg_mass_apply": (i, [vp, i, i, vp, vp, d]),
        "sipg_inverse_mass_apply": (i, [vp, i, i, vp, vp, d]),
        "sipg_default_picard_opts": (None, [P(PicardOpts)]),
        "sipg_picard_solve": (i, [vp, P(Rheology), vp, vp, P(PicardOpts), P(PicardStats)]),
        "sipg_ff_convert": (i, [vp, vp, vp, vp, i64]),
        "sipg_default_step_opts": (None, [P(StepOpts)]),
        "sipg_step_init": (i, [vp, vp, vp]),
        "sipg_step": (i, [vp, P(Rheology), P(StepOpts), P(StepStats)]),
        "sipg_step_field": (i, [vp, i, vp]),
        "sipg_cfl_dt": (i, [vp, vp, d, P(d)]),
        "sipg_convective_apply": (i, [vp, vp, vp, vp]),
        "sipg_projection_rhs": (i, [vp, vp, vp]),
        "sipg_viscous_wall_rhs": (i, [vp, vp, vp]),
        "sipg_solve_convective": (i, [vp, vp, vp, vp, vp, P(SolveOpts), i, P(SolveStats)]),
        "sipg_convective_lin_apply": (i, [vp, vp, vp, vp, vp, vp]),
        "sipg_penalty_tau": (i, [vp, vp, d, d, d, vp, vp]),
        "sipg_penalty_apply": (i, [vp, vp, vp, vp, vp]),
        "sipg_penalty_wall_rhs": (i, [vp, vp, vp, vp]),
        "sipg_penalty_step": (i, [vp, vp, vp, d, d, d, d, i, vp, P(i), P(d)]),
        "sipg_boundary_faces": (i, [vp, P(i), vp, vp]),
        "sipg_rhs_manufactured": (i, [vp, i, vp]),
        "sipg_topology_tables": (i, [i, i, i, vp, vp, P(i), P(i), vp, vp]),
        "sipg_coarsen_mask": (i, [i, i, i, vp, vp]),
        "sipg_level_plan": (i, [P(MeshDesc), P(Opts), i, i, P(i), vp]),
        "sipg_alu_peak": (i, [i, P(d)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
