"""Failure detection on the GPU, without faulting it.

* Bounded waits of the tensor-core kernels: a test switch makes the first
  trailing-update CTA withhold one operand copy, so the tensor-core issuer's
  wait for it can only end by its limit (set to a few milliseconds).  The
  call must report BEOR_ETIMEOUT and name a role wait as the one that gave
  up first (the issuer waiting for the withheld operands, the epilogue
  waiting for that tile's accumulators, or the producer waiting for the
  withheld slot to be released: all three wait on it, and a waiting thread
  may be suspended between checks of its deadline, so which one fires first
  is not fixed), the context must then refuse work (BEOR_ESTATE), and a
  fresh context must evaluate correctly afterwards.
* A non-finite phi passed in device memory marks that point only (status -2,
  lnL NaN); the other points of the batch are unaffected.
"""

import numpy as np
import pytest

from gpu_common import make_like, oracle_eval, phis

pytestmark = pytest.mark.gpu

ETIMEOUT, ESTATE = -4, -5
ROLE_WAIT_CODES = (11, 12, 13, 14)   # producer, issuer (operands), issuer (accumulators), epilogue


def test_bounded_wait_gives_up_and_reports():
    import paper_2501_12928_gb300 as P

    try:
        P.set_wait_test(True, 5.0)
        lk = make_like(P, "C0", "mixed")
        ph = phis("C0", 4)
        with pytest.raises(P.BeorError) as ei:
            lk.lnl(ph)
        assert f"({ETIMEOUT})" in str(ei.value)
        assert lk.stats()["device_error"] in ROLE_WAIT_CODES
        with pytest.raises(P.BeorError) as ei:
            lk.lnl(ph)
        assert f"({ESTATE})" in str(ei.value)
        lk.close()
    finally:
        P.set_wait_test(False, 0.0)
    # a fresh context on the same device works and matches the oracle
    lk = make_like(P, "C0", "mixed")
    got, st = lk.lnl(ph)
    assert np.all(st == 0), st
    ref = np.array([oracle_eval("C0", p)["lnl"] for p in ph])
    assert np.abs(got - ref).max() <= 1e-2
    lk.close()


def test_short_wait_limit_alone_does_not_fire():
    """A short role-wait limit without a withheld copy still completes: the
    waits of a normal evaluation are far shorter than 50 ms."""
    import paper_2501_12928_gb300 as P

    try:
        P.set_wait_test(False, 50.0)
        lk = make_like(P, "C0", "mixed")
        ph = phis("C0", 4)
        got, st = lk.lnl(ph)
    finally:
        P.set_wait_test(False, 0.0)
    assert np.all(st == 0)
    ref = np.array([oracle_eval("C0", p)["lnl"] for p in ph])
    assert np.abs(got - ref).max() <= 1e-2
    lk.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_phi_on_device_marks_only_that_point(precision):
    import torch

    import paper_2501_12928_gb300 as P

    lk = make_like(P, "C0", precision)
    ph = phis("C0", 6)
    bad = ph.copy()
    bad[1, 2] = np.nan
    bad[4, 0] = np.inf
    dphi = torch.tensor(bad, dtype=torch.float64, device="cuda")
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    st = torch.empty(6, dtype=torch.int32, device="cuda")
    lk.lnl(dphi, out=out, status=st)
    torch.cuda.synchronize()
    got, sts = out.cpu().numpy(), st.cpu().numpy()
    assert sts[1] == -2 and sts[4] == -2, sts
    assert np.isnan(got[1]) and np.isnan(got[4])
    tol = 1e-10 if precision == "fp64" else 1e-2
    for b in (0, 2, 3, 5):
        assert sts[b] == 0
        ref = oracle_eval("C0", ph[b])["lnl"]
        err = abs(got[b] - ref)
        assert err <= (tol * abs(ref) if precision == "fp64" else tol), (b, err)
    # host phi with a non-finite value is an argument error
    with pytest.raises(P.BeorError):
        lk.lnl(bad)
    lk.close()
