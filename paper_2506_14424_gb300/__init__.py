"""GB300 (sm_103a) matrix-free SIPG operators and CG / hp-multigrid solver.

Implements the hot path of arXiv 2506.14424 (Schussnig, Fehn, Pacheco,
Kronbichler): the variable-viscosity viscous operator -div(2 nu eps(u)) and the
pressure Poisson operator, discretised with the symmetric interior penalty
discontinuous Galerkin method on hexahedra and evaluated matrix-free by sum
factorisation, inside an FP64 conjugate-gradient solver preconditioned by a
Chebyshev-smoothed hp-multigrid V-cycle in FP32.

``Context`` (``api.py``) wraps the C ABI of ``include/sipg.h``;
``build.build()`` compiles ``libsipg.so``; ``inputs`` holds the seeded
synthetic workloads. ``Context`` is imported lazily so that ``inputs`` can be
used without loading torch.
"""


def __getattr__(name):
    if name in ("Context", "SipgError", "Server", "estimate_bytes", "alu_peak"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
