"""The schedule autotuner (beor_autotune): every candidate schedule does the
same operations on every tile, so the chosen schedule's factors and
log-determinants equal the default schedule's bit for bit; the choice is
written to and read back from the cache file."""

import json

import numpy as np
import pytest

from gpu_common import make_like, oracle_eval, phis

pytestmark = pytest.mark.gpu


def test_autotuned_schedule_is_bitwise_default(tmp_path):
    import paper_2501_12928_gb300 as P

    # two instruments of uneven size in one batch (aligned ends matter)
    likes = [make_like(P, "C0", "mixed"), make_like(P, "C1", "mixed")]
    ph = [phis("C0", 4), phis("C1", 4)]
    Bs = [4, 4]
    try:
        P.set_schedule(likes, Bs, None)
        ref_out, ref_st = P.lnl_multi(likes, ph)
        ref_L = likes[1].factor(2)
        ref_terms = [lk.terms(4) for lk in likes]

        cache = str(tmp_path / "tune.jsonl")
        res = P.autotune(likes, ph, reps=1, cache_path=cache)
        print(res)
        assert P.get_schedule(likes, Bs) == res["schedule"]
        assert res["ms_per_eval"] > 0 and res["ms_default"] >= res["ms_per_eval"]
        out, st = P.lnl_multi(likes, ph)
        for a, b in zip(st, ref_st):
            assert np.all(a == 0) and np.all(b == 0)
        np.testing.assert_array_equal(likes[1].factor(2), ref_L)
        for lk, rt in zip(likes, ref_terms):
            t = lk.terms(4)
            np.testing.assert_array_equal(t["logdet_sigma"], rt["logdet_sigma"])
            np.testing.assert_array_equal(t["logdet_phi"], rt["logdet_phi"])
        for a, b in zip(out, ref_out):
            assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()
        # against the oracle as well
        for s, name in enumerate(("C0", "C1")):
            ref = oracle_eval(name, ph[s][0])["lnl"]
            assert abs(out[s][0] - ref) <= 1e-2

        # the cache holds one entry for this shape; a second call reads it back
        lines = [json.loads(x) for x in open(cache)]
        assert len(lines) == 1 and lines[0]["lookahead"] == res["schedule"]["lookahead"]
        P.set_schedule(likes, Bs, None)
        res2 = P.autotune(likes, ph, reps=1, cache_path=cache)
        assert res2["schedule"] == res["schedule"]
        assert len(open(cache).readlines()) == 1
    finally:
        P.set_schedule(likes, Bs, None)


def test_every_schedule_gives_the_same_factor():
    import paper_2501_12928_gb300 as P

    likes = [make_like(P, "C0", "mixed"), make_like(P, "C1", "mixed")]
    ph = [phis("C0", 2, stream=5), phis("C1", 2, stream=5)]
    Bs = [2, 2]
    scheds = [dict(lookahead=1, rest_ctas=0, col_ctas=0, align_ends=1, reserve_diag=0),
              dict(lookahead=1, rest_ctas=100, col_ctas=37, align_ends=0, reserve_diag=0),
              dict(lookahead=1, rest_ctas=0, col_ctas=0, align_ends=1, reserve_diag=1),
              dict(lookahead=0, rest_ctas=0, col_ctas=0, align_ends=0, reserve_diag=0),
              dict(lookahead=0, rest_ctas=64, col_ctas=5, align_ends=1, reserve_diag=1)]
    try:
        facs, dets = [], []
        for sc in scheds:
            P.set_schedule(likes, Bs, sc)
            assert P.get_schedule(likes, Bs) == sc
            _, st = P.lnl_multi(likes, ph)
            assert all(np.all(x == 0) for x in st)
            facs.append(likes[1].factor(1))
            dets.append(likes[1].terms(2)["logdet_sigma"])
        for f, d in zip(facs[1:], dets[1:]):
            np.testing.assert_array_equal(f, facs[0])
            np.testing.assert_array_equal(d, dets[0])
    finally:
        P.set_schedule(likes, Bs, None)
