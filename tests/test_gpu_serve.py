"""Continuous-batching server on the GPU (the serving pattern of the solver).

* served solutions solve the oracle's own system: for a mix of meshes, degrees
  2..5, viscosity contrasts 1..1e4 and right-hand sides made by the oracle
  (host and device b) or by the server (buoyancy M f, b = A u*), the oracle
  recomputes ||b - A_ref x|| <= 1e-8 (1 + 1e-6) ||b|| with its assembled forms;
* the served FP64 solve agrees with a stand-alone Context.solve of the same
  system to the solve tolerance;
* a request's solution is bitwise the same alone and batched with others of
  different mesh size and degree (the batched apply runs the same per-cell
  code, all reductions are deterministic), with either Krylov operator;
* admission by HBM budget: a request that can never fit is rejected with
  SIPG_ERR_NOMEM, and a budget that holds one context at a time still serves
  every request.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import viscosity  # noqa: E402
from oracle.mass import apply_mass  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, Server, estimate_bytes, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
GiB = 1 << 30
RTOL = 1e-8


def _sinker(seed, contrast):
    return inputs.sinker(seed=seed, count=8, radius=0.15, nu_max=contrast)


def _oracle(n, k, rh):
    S = SIPG(BoxMesh(n, n, n), k, 3)
    nc, nf = S.viscosity_at_points(rh)
    return S, nc, nf


def _buoyancy_ref(S, rh):
    """b = M f with f the nodal interpolant of -e_z chi (sphere indicator, ties inside)."""
    def f(p):
        chi = viscosity.sinker_field(p, rh['centers'], rh['radius'], 1.0, 0.0)
        return np.stack([0 * chi, 0 * chi, -chi], axis=1)
    return apply_mass(S, S.interpolate(f))


def test_served_solutions_solve_the_oracle_system():
    cases = [(4, 2, _sinker(21, 1.0), "host"),
             (3, 3, _sinker(22, 1e2), "device"),
             (2, 4, _sinker(23, 1e4), "buoyancy"),
             (2, 5, _sinker(24, 1e2), "host")]
    refs, ids, keep = [], [], []
    srv = Server(8 * GiB, max_slots=4)
    for i, (n, k, rh, kind) in enumerate(cases):
        S, nc, nf = _oracle(n, k, rh)
        if kind == "buoyancy":
            b = _buoyancy_ref(S, rh)
            rhs = "buoyancy"
        else:
            b = S.apply(inputs.uniform_vector(S.n_dofs, seed=60 + i), nc, nf)
            rhs = b if kind == "host" else torch.tensor(b, device="cuda")
            keep.append(rhs)
        refs.append((S, nc, nf, b))
        ids.append(srv.submit(n, k, rh, rtol=RTOL, seed=70 + i, keep_solution=True, rhs=rhs))
    srv.drain(300)
    for (S, nc, nf, b), rid in zip(refs, ids):
        res, x = srv.poll(rid)
        assert res["status"] == 0, res
        assert np.isnan(res["err_vs_ustar"])
        r_ref = np.linalg.norm(b - S.apply(x, nc, nf)) / np.linalg.norm(b)
        assert r_ref <= RTOL * (1 + 1e-6), (res, r_ref)
        assert abs(r_ref - res["rel_residual"]) <= 1e-10
    srv.close()


def test_served_solution_matches_a_standalone_solve():
    rh = _sinker(25, 1e2)
    S, nc, nf = _oracle(3, 3, rh)
    b = S.apply(inputs.uniform_vector(S.n_dofs, seed=80), nc, nf)
    srv = Server(8 * GiB, max_slots=2)
    rid = srv.submit(3, 3, rh, rtol=1e-10, keep_solution=True, rhs=b)
    srv.drain(120)
    res, x = srv.poll(rid)
    srv.close()
    assert res["status"] == 0
    ctx = Context(3, 3, 3, 3)
    ctx.set_viscosity(rh)
    xs, st = ctx.solve("viscous", torch.tensor(b, device="cuda"), rtol=1e-10, precond="mg")
    ctx.close()
    xs = xs.cpu().numpy()
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)


@pytest.mark.parametrize("arith", ["f64", "f64ff"])
def test_result_is_the_same_alone_and_in_the_mix(arith):
    srv = Server(8 * GiB, max_slots=4, krylov_arith=arith)
    a = srv.submit(6, 3, _sinker(5, 1e2), seed=11, keep_solution=True)
    srv.drain(120)
    ra, xa = srv.poll(a)
    assert ra["status"] == 0 and ra["rel_residual"] <= 1e-8
    ids = [srv.submit(4, 2, _sinker(6, 1.0), seed=12, keep_solution=True),
           srv.submit(6, 3, _sinker(5, 1e2), seed=11, keep_solution=True),
           srv.submit(8, 4, _sinker(7, 1e4), seed=13, keep_solution=True),
           srv.submit(4, 5, _sinker(8, 1e2), seed=14, keep_solution=True, rhs="buoyancy")]
    srv.drain(300)
    res = [srv.poll(i) for i in ids]
    for j, (r, x) in enumerate(res):
        assert r["status"] == 0, r
        assert r["rel_residual"] <= 1e-8
        if j != 3:
            assert r["err_vs_ustar"] < 1e-4
    rb, xb = res[1]
    assert rb["iterations"] == ra["iterations"]
    assert np.array_equal(xa, xb)
    srv.close()


def test_admission_by_budget():
    need = estimate_bytes(6, 3)
    srv = Server(int(need * 1.2) + 64 * 3 * 6 ** 3 * 4 ** 3, max_slots=4)
    big = srv.submit(12, 4, _sinker(1, 1.0), seed=1)          # never fits
    small = [srv.submit(6, 3, _sinker(2 + i, 1e2), seed=20 + i) for i in range(3)]
    srv.drain(300)
    rbig, _ = srv.poll(big)
    assert rbig["status"] == -3
    for i in small:
        r, _ = srv.poll(i)
        assert r["status"] == 0 and r["rel_residual"] <= 1e-8
    srv.close()


def test_submit_rejects_velocity_dependent_laws_and_missing_rhs():
    srv = Server(1 * GiB, max_slots=1)
    with pytest.raises(Exception):
        srv.submit(4, 2, inputs.carreau_blood_like())
    srv.close()
