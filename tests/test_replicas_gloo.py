"""Replica path on two CPU ranks (gloo): sharding, gather of results, max
timing, and a rank that dies before the gather (the survivor gets an error
within the process-group timeout instead of hanging)."""

import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2501_12928_gb300.replicas import shard_bounds


def test_shard_bounds_cover():
    for n in (0, 1, 5, 16, 17):
        for w in (1, 2, 3, 4):
            seen = []
            for r in range(w):
                lo, hi = shard_bounds(n, r, w)
                seen.extend(range(lo, hi))
            assert seen == list(range(n))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _loglike(phi):
    # the oracle on a tiny problem: per-point lnL, status 0
    import oracle as O
    from synth.instrument import random_problem
    p = random_problem(12, 5, 2, 0)
    M = O.herm_dense(p["T"], p["noise_var"])
    db = O.dbar_dense(p["T"], p["noise_var"], p["d"])
    return np.array([O.evaluate(M, db, p["kbin"], x, 3.0)["lnl"] for x in phi]), np.zeros(len(phi), np.int32)


def _worker(rank, world, port, mode, q):
    import torch.distributed as dist
    from paper_2501_12928_gb300.replicas import evaluate_sharded, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    phi = np.random.default_rng(0).uniform(-2, 2, (7, 2))
    try:
        if mode == "die" and rank == 1:
            os._exit(0)                    # leaves between steps, nothing in flight
        vals, st = evaluate_sharded(_loglike, phi)
        t = max_over_ranks(0.5 + rank)
        q.put((rank, "ok", vals.tolist(), st.tolist(), t))
    except Exception as e:                 # noqa: BLE001
        q.put((rank, "error", type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:                  # noqa: BLE001
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = []
    for p in procs:
        p.join(timeout=120)
        assert not p.is_alive()
    while not q.empty():
        out.append(q.get())
    return sorted(out)


def test_two_rank_gather_matches_single_process():
    res = _run("ok")
    assert len(res) == 2
    ref, _ = _loglike(np.random.default_rng(0).uniform(-2, 2, (7, 2)))
    for rank, status, vals, st, t in res:
        assert status == "ok"
        assert np.allclose(vals, ref, rtol=0, atol=1e-12)
        assert st == [0] * 7
        assert t == 1.5


def test_dead_rank_is_detected():
    res = _run("die")
    assert len(res) == 1 and res[0][0] == 0 and res[0][1] == "error"
