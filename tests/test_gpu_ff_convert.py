"""Float-float loads and stores of the SIPG_F64_FF kernels, bit for bit.

The kernels split each binary64 value into hi = RN(x), lo = RN(x - hi) (binary32,
round to nearest even) and join a result as hi + lo rounded to binary64. The
expected bits come from numpy's IEEE casts, which define those roundings; the
values cover random magnitudes over 2^-100..2^130, exact ties of both
roundings and every special class (zeros, subnormals, infinities, NaN).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_14424_gb300 import Context  # noqa: E402

pytestmark = pytest.mark.gpu


def _values():
    rng = np.random.default_rng(0)
    v = [rng.uniform(-1, 1, 200000),
         rng.standard_normal(200000) * 2.0 ** rng.integers(-100, 130, 200000)]
    ties = []
    for base in [1.0, 1.5, 3.0, 1.0 + 2 ** -23, 1.0 + 2 ** -22, 0.75]:
        ties += [base + 2 ** -24, base - 2 ** -25, base + 2 ** -24 + 2 ** -50, base + 3 * 2 ** -24,
                 base + 2 ** -47, base + 2 ** -48 + 2 ** -52, base + 2 ** -48, base + 3 * 2 ** -48]
    ties = np.array(ties)
    edges = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, 1e-300, 2.0 ** -70, 2.0 ** -70 * (1 - 2 ** -53),
                      2.0 ** -71, 2.0 ** 127 * (1 - 2 ** -53), 2.0 ** 127, 3.4028234663852886e38,
                      3.4028235677973366e38, 1e300, -1e300, np.inf, -np.inf, np.nan, 1.0, -1.0,
                      2.0 ** -126, 2.0 ** -149, 1.0 - 2 ** -53])
    return np.concatenate(v + [ties, -ties, edges])


def test_split_and_join_bit_exact():
    ctx = Context(1, 1, 1, 2)
    x = _values()
    hilo, back = ctx.ff_convert(torch.tensor(x, device="cuda"))
    hilo, back = hilo.cpu().numpy(), back.cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        hi = x.astype(np.float32)
        lo = (x - hi.astype(np.float64)).astype(np.float32)
        joined = hi.astype(np.float64) + lo.astype(np.float64)
    nan = np.isnan(x)
    assert np.array_equal(hilo[~nan, 0].view(np.uint32), hi[~nan].view(np.uint32))
    lo_ok = np.isnan(lo) & np.isnan(hilo[:, 1]) | (hilo[:, 1].view(np.uint32) == lo.view(np.uint32))
    assert lo_ok[~nan].all()
    j_ok = (np.isnan(joined) & np.isnan(back)) | (back.view(np.uint64) == joined.view(np.uint64))
    assert j_ok[~nan].all()
    assert np.isnan(hilo[nan, 0]).all() and np.isnan(back[nan]).all()
    ctx.close()
