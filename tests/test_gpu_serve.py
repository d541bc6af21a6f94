"""Continuous-batching server on the GPU (the serving pattern of the solver).

* every request converges to rtol 1e-8 (true residual), in the mix as alone;
* a request's solution is bitwise the same alone and batched with others of
  different mesh size and degree (the batched apply runs the same per-cell
  code, all reductions are deterministic);
* admission by HBM budget: a request that can never fit is rejected with
  SIPG_ERR_NOMEM, and a budget that holds one context at a time still serves
  every request.
"""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2506_14424_gb300 import Server, estimate_bytes, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
GiB = 1 << 30


def _sinker(seed, contrast):
    return inputs.sinker(seed=seed, count=8, radius=0.15, nu_max=contrast)


def test_result_is_the_same_alone_and_in_the_mix():
    srv = Server(8 * GiB, max_slots=4)
    a = srv.submit(6, 3, _sinker(5, 1e2), seed=11, keep_solution=True)
    srv.drain(120)
    ra, xa = srv.poll(a)
    assert ra["status"] == 0 and ra["rel_residual"] <= 1e-8
    ids = [srv.submit(4, 2, _sinker(6, 1.0), seed=12, keep_solution=True),
           srv.submit(6, 3, _sinker(5, 1e2), seed=11, keep_solution=True),
           srv.submit(8, 4, _sinker(7, 1e4), seed=13, keep_solution=True),
           srv.submit(4, 5, _sinker(8, 1e2), seed=14, keep_solution=True)]
    srv.drain(300)
    res = [srv.poll(i) for i in ids]
    for r, x in res:
        assert r["status"] == 0, r
        assert r["rel_residual"] <= 1e-8
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
