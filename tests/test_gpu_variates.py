"""The exponential variates E = -ln u that every kernel draws from a Philox word, computed with the
library's logarithm, against the float64 logarithm of the same uniforms, for all 2^23 uniforms the
map u = ((x >> 9) + 1/2) 2^-23 can produce."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_exponential_variates_of_every_uniform_are_accurate():
    from paper_2602_19775_gb300 import ssa
    m = np.arange(1 << 23, dtype=np.uint32)
    E = ssa.exp_variates(m << np.uint32(9)).cpu().numpy().astype(np.float64)
    ref = -np.log((m.astype(np.float64) + 0.5) * 2.0 ** -23)
    ulp = 2.0 ** (np.floor(np.log2(ref)) - 23)
    err = np.abs(E - ref) / ulp
    assert err.max() <= 1.5, (err.max(), int(np.argmax(err)))  # logf: within one ulp, plus the ulp boundary
    assert np.all(E > 0) and np.all(np.isfinite(E))
