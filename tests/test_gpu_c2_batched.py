"""The 3280-mode instrument with B = 64 points in one batched mixed-precision
evaluation: every status is 0, sampled points agree with the oracle
(|dlnL| <= 1e-2), and each sampled point evaluated alone gives the same lnL
to within the rounding of the float64 residual, which sums with atomics
(batch invariance)."""

import numpy as np
import pytest

from tests.gpu_common import make_like, oracle_eval, phis

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_c1_b64_batched_sampled_parity():
    import paper_2501_12928_gb300 as P

    lk = make_like(P, "C1", precision="mixed")
    ph = phis("C1", 64, stream=61)
    got, st = lk.lnl(ph)
    assert np.all(st == 0), st
    for b in (0, 31, 63):
        ref = oracle_eval("C1", ph[b])["lnl"]
        print("C1 B=64 point", b, "|dlnL|", abs(got[b] - ref))
        assert abs(got[b] - ref) <= 1e-2
        single, s1 = lk.lnl(ph[b:b + 1])
        assert s1[0] == 0
        assert abs(single[0] - got[b]) <= 1e-3, (b, single[0], got[b])
