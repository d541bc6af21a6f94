"""The allocation-free apply entry point against the ordinary one (GPU).

sipg_apply_host_static exists for callers that must not let a library call
allocate device memory; it stages the host vectors in a fixed device array
instead of context-owned buffers. This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2506_14424_gb300 import Context, SipgError, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_static_apply_matches_apply_host_on_two_calls():
    ctx = Context(4, 3, 2, 3, bc_velocity="DDNDDD")
    ctx.set_viscosity({'law': 'analytic'})
    n = ctx.n_dofs("viscous")
    for seed in (41, 42):  # two calls in a row through the shared staging area
        x = inputs.uniform_vector(n, seed=seed)
        y_ref = ctx.apply_host("viscous", x)
        y = ctx.apply_host_static("viscous", x)
        assert _rel(y, y_ref) <= TOL64
    xp = inputs.uniform_vector(ctx.n_dofs("poisson"), seed=43)
    assert _rel(ctx.apply_host_static("poisson", xp), ctx.apply_host("poisson", xp)) <= TOL64
    ctx.close()


def test_static_apply_rejects_oversized_vectors():
    ctx = Context(12, 12, 12, 4)  # 648,000 velocity DoFs > 524,288
    ctx.set_viscosity({'law': 'constant', 'nu': 1.0})
    with pytest.raises(SipgError) as ei:
        ctx.apply_host_static("viscous", np.zeros(ctx.n_dofs("viscous")))
    assert ei.value.code == -1 and "static staging area" in str(ei.value)
    ctx.close()
