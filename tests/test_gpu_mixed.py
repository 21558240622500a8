"""GPU mixed-precision path (bf16 slice products on tcgen05, double-float
working matrix, float64 diagonal blocks and refinement) against the CPU oracle.

Tolerances: |lnL - lnL_oracle| <= 1e-2 absolute and
||abar - abar_oracle|| / ||abar_oracle|| <= 1e-6.
"""

import numpy as np
import pytest

import oracle as O
from synth.instrument import random_problem
from tests.gpu_common import make_like, oracle_eval, phis

pytestmark = pytest.mark.gpu

ATOL_LNL = 1e-2
RTOL_ABAR = 1e-6


@pytest.fixture(scope="module")
def P():
    import paper_2501_12928_gb300 as P
    return P


def test_mixed_C0(P):
    lk = make_like(P, "C0", precision="mixed")
    ph = phis("C0", 16, stream=41)
    got, st = lk.lnl(ph)
    ref = np.array([oracle_eval("C0", p)["lnl"] for p in ph])
    assert np.all(st == 0), st
    err = np.abs(got - ref)
    print("C0 mixed max |dlnL|", err.max(), lk.stats())
    assert err.max() <= ATOL_LNL


def test_mixed_posterior_mean_C0(P):
    lk = make_like(P, "C0", precision="mixed")
    for p in phis("C0", 3, stream=43):
        a, st = lk.posterior_mean(p)
        ref = oracle_eval("C0", p)["abar"]
        assert st == 0
        assert np.linalg.norm(a - ref) <= RTOL_ABAR * np.linalg.norm(ref)


@pytest.mark.parametrize("nvis,n,nk", [(12, 5, 2), (300, 130, 3), (400, 383, 5), (700, 640, 4)])
def test_mixed_random_shapes(P, nvis, n, nk):
    p = random_problem(nvis, n, nk, seed=n + 1)
    lk = P.Likelihood("mixed")
    lk.set_T(p["T"], p["kbin"], nk, 2.0)
    lk.set_data(p["d"], p["noise_var"])
    lk.precompute()
    M = O.herm_dense(p["T"], p["noise_var"])
    db = O.dbar_dense(p["T"], p["noise_var"], p["d"])
    ph = np.random.default_rng(n).uniform(-2, 2, (4, nk))
    got, st = lk.lnl(ph)
    for i in range(4):
        r = O.evaluate(M, db, p["kbin"], ph[i], 2.0)
        assert st[i] == 0 and abs(got[i] - r["lnl"]) <= ATOL_LNL, (i, got[i], r["lnl"])
    a, st0 = lk.posterior_mean(ph[0])
    ref = O.evaluate(M, db, p["kbin"], ph[0], 2.0)["abar"]
    assert np.linalg.norm(a - ref) <= RTOL_ABAR * np.linalg.norm(ref)


def test_mixed_matches_fp64_gpu_C0(P):
    a = make_like(P, "C0", precision="mixed")
    b = make_like(P, "C0", precision="fp64")
    ph = phis("C0", 8, stream=47)
    la, _ = a.lnl(ph)
    lb, _ = b.lnl(ph)
    assert np.abs(la - lb).max() <= ATOL_LNL


@pytest.mark.slow
def test_mixed_and_fp64_C1_full_size(P):
    """The 3280-mode instrument at full size: mixed |dlnL| <= 1e-2, abar rel
    <= 1e-6; float64 GPU 1e-10 relative."""
    ph = phis("C1", 2, stream=51)
    refs = [oracle_eval("C1", p) for p in ph]
    lm = make_like(P, "C1", precision="mixed")
    got, st = lm.lnl(ph)
    assert np.all(st == 0)
    errs = np.abs(got - np.array([r["lnl"] for r in refs]))
    print("C1 mixed |dlnL|", errs, lm.stats()["resid_rel_max"])
    assert errs.max() <= ATOL_LNL
    a, _ = lm.posterior_mean(ph[0])
    assert np.linalg.norm(a - refs[0]["abar"]) <= RTOL_ABAR * np.linalg.norm(refs[0]["abar"])
    lf = make_like(P, "C1", precision="fp64")
    gf, sf = lf.lnl(ph)
    assert np.all(sf == 0)
    assert np.all(np.abs(gf - np.array([r["lnl"] for r in refs])) <= 1e-10 * np.abs([r["lnl"] for r in refs]))


def _uneven_batch(P):
    likes, refs, phs = [], [], []
    for nvis, n, nk in ((700, 640, 4), (400, 383, 3), (1300, 1100, 5)):
        p = random_problem(nvis, n, nk, seed=n + 7)
        lk = P.Likelihood("mixed")
        lk.set_T(p["T"], p["kbin"], nk, 2.0)
        lk.set_data(p["d"], p["noise_var"])
        lk.precompute()
        ph = np.random.default_rng(n + 3).uniform(-2, 2, (3, nk))
        M = O.herm_dense(p["T"], p["noise_var"])
        db = O.dbar_dense(p["T"], p["noise_var"], p["d"])
        refs.append([O.evaluate(M, db, p["kbin"], q, 2.0)["lnl"] for q in ph])
        likes.append(lk)
        phs.append(ph)
    return likes, phs, refs


def test_lookahead_schedule_is_bitwise_in_order(P):
    """The look-ahead schedule (split trailing update on two streams, dynamic
    tile order) applies the same operations to every tile as the in-order
    schedule: the Cholesky factors agree bit for bit, with and without
    profiling events, on a batch of uneven sizes (5, 3 and 9 block steps).
    lnL agrees to rounding (the float64 refinement residual sums tiles with
    atomics, in no fixed order)."""
    likes, phs, refs = _uneven_batch(P)
    runs = {}
    try:
        for la in (True, False):
            for prof in (False, True):
                P.set_lookahead(la)
                P.set_profiling(prof)
                for _ in range(2):   # first call runs directly, the second replays the graph
                    outs, sts = P.lnl_multi(likes, phs)
                    assert all(np.all(s == 0) for s in sts)
                    facs = [lk.factor(b) for lk in likes for b in (0, 2)]
                    runs.setdefault((la, prof), []).append((np.concatenate(outs), facs))
    finally:
        P.set_lookahead(True)
        P.set_profiling(False)
    base, base_f = runs[(False, False)][0]
    for key, vals in runs.items():
        for v, f in vals:
            for a, b in zip(f, base_f):
                assert np.array_equal(a, b), key
            assert np.allclose(v, base, rtol=1e-13, atol=0), (key, v - base)
    err = np.abs(base - np.concatenate(refs))
    assert err.max() <= ATOL_LNL, err
    st = likes[0].stats()
    assert st["n_class"]["trail"] > 0 and st["ms_class"]["trail"] > 0


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_ragged_batches_across_sets(P, precision):
    """Uneven sizes (1, 3 and 9 block steps) with ragged batch sizes per set
    (1, 17 and 5 points: the 17 span two 16-point residual work groups),
    every point against the oracle."""
    specs = ((90, 70, 2, 1), (400, 383, 3, 17), (1300, 1100, 5, 5))
    likes, phs, refs = [], [], []
    for nvis, n, nk, B in specs:
        p = random_problem(nvis, n, nk, seed=n + 11)
        lk = P.Likelihood(precision)
        lk.set_T(p["T"], p["kbin"], nk, 2.0)
        lk.set_data(p["d"], p["noise_var"])
        lk.precompute()
        ph = np.random.default_rng(n + 5).uniform(-2, 2, (B, nk))
        M = O.herm_dense(p["T"], p["noise_var"])
        db = O.dbar_dense(p["T"], p["noise_var"], p["d"])
        refs.append(np.array([O.evaluate(M, db, p["kbin"], q, 2.0)["lnl"] for q in ph]))
        likes.append(lk)
        phs.append(ph)
    outs, sts = P.lnl_multi(likes, phs)
    for o, st, r in zip(outs, sts, refs):
        assert np.all(st == 0), st
        if precision == "fp64":
            assert np.all(np.abs(o - r) <= 1e-10 * np.abs(r)), np.abs(o - r) / np.abs(r)
        else:
            assert np.abs(o - r).max() <= ATOL_LNL, np.abs(o - r)


def test_async_slots_match_synchronous(P):
    """Two batches in flight on two slots and two streams give the same lnL
    as the synchronous call (the factorisation is deterministic; the float64
    residual sums tiles in no fixed order), twice in a row."""
    import torch
    likes, phs, refs = _uneven_batch(P)
    sync_out, _ = P.lnl_multi(likes, phs)
    dev_phi = [torch.tensor(p, dtype=torch.float64, device="cuda") for p in phs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [[torch.empty(len(p), dtype=torch.float64, device="cuda") for p in phs] for _ in range(2)]
    sts = [[torch.empty(len(p), dtype=torch.int32, device="cuda") for p in phs] for _ in range(2)]
    Bs = [len(p) for p in phs]
    for _ in range(2):
        for slot in (0, 1):
            P.lnl_multi_async(likes, dev_phi, outs[slot], sts[slot], slot, streams[slot])
        for slot in (0, 1):
            P.lnl_multi_wait(likes, Bs, slot, streams[slot])
            got = np.concatenate([o.cpu().numpy() for o in outs[slot]])
            assert all(int((s != 0).sum()) == 0 for s in sts[slot])
            assert np.allclose(got, np.concatenate(sync_out), rtol=1e-12, atol=0)
    with pytest.raises(P.BeorError):      # host buffers are rejected
        P.lnl_multi_async(likes, [np.ascontiguousarray(p) for p in phs], outs[0], sts[0], 0, streams[0])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_singular_point_is_isolated(P, precision):
    """A point at which Sigma is singular gets status j > 0 and lnL = -inf,
    and the other points of the batch are unaffected.  Columns 0 and 1 of T
    are equal (2 at visibility 0, unit noise variance there), so
    M_00 = M_01 = M_11 = 4 exactly; phi = 400 makes Phi^-1 of their k bin
    underflow to 0, and the second pivot is 4 - 2 * 2 = 0 exactly in any
    correctly rounded arithmetic: status 2, the oracle's too.  With 300
    modes the failed point is carried through three block steps."""
    p = random_problem(400, 300, 3, seed=5)
    T, nv, kbin = p["T"].copy(), p["noise_var"].copy(), p["kbin"].copy()
    T[:, 0] = 0.0
    T[0, 0] = 2.0
    T[:, 1] = T[:, 0]
    nv[0] = 1.0
    kbin[1] = 0
    lk = P.Likelihood(precision)
    lk.set_T(T, kbin, 3, 2.0)
    lk.set_data(p["d"], nv)
    lk.precompute()
    ph = np.array([[0.3, -0.5, 1.0], [400.0, -0.5, 1.0], [-1.0, 0.7, 0.2]])
    got, st = lk.lnl(ph)
    M = O.herm_dense(T, nv)
    db = O.dbar_dense(T, nv, p["d"])
    ref = [O.evaluate(M, db, kbin, x, 2.0) for x in ph]
    assert [r["status"] for r in ref] == [0, 2, 0]
    assert list(st) == [0, 2, 0], st
    assert got[1] == -np.inf
    tol = ATOL_LNL if precision == "mixed" else 1e-10 * max(abs(ref[0]["lnl"]), abs(ref[2]["lnl"]))
    for i in (0, 2):
        assert abs(got[i] - ref[i]["lnl"]) <= tol, (i, got[i], ref[i]["lnl"])


def test_empty_batch_is_rejected(P):
    """B = 0 is an argument error (BEOR_EINVAL), not an empty launch."""
    lk = make_like(P, "C0", precision="mixed")
    with pytest.raises(P.BeorError, match=r"\(-1\)"):
        lk.lnl(np.zeros((0, 4)))

