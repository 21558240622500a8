"""The bounds-checked build (BEOR_BOUNDS_CHECK; the stand-in for a device
memory checker): the factorisation, solve and residual kernels check their
packed-tile, slice-plane, vector and tensor-map indices, record the first
failed check and skip the access.  Evaluations of several shapes -- odd
sizes with ragged tiles, an uneven batch of two instruments, the float64
path, the posterior mean -- must report no failed check and still match the
oracle.  Runs in a child process that loads _build/libbeor_checked.so."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import oracle as O
import paper_2501_12928_gb300 as P
from paper_2501_12928_gb300 import beor as B
from gpu_common import make_like, oracle_eval, phis
from synth.instrument import random_problem

out = {"build_info": B._lib().beor_build_info(), "cases": []}
def record(name, lk, err):
    out["cases"].append({"name": name, "bounds": lk.stats()["bounds_error"], "err": float(err)})

for prec in ("fp64", "mixed"):
    lk = make_like(P, "C0", prec)
    ph = phis("C0", 5)
    got, st = lk.lnl(ph)
    ref = np.array([oracle_eval("C0", p)["lnl"] for p in ph])
    record("C0 " + prec, lk, np.abs(got - ref).max())
# odd shapes: ragged last tile, and fewer visibilities than a tile
for n_vis, n_model in ((300, 131), (90, 260)):
    p = random_problem(n_vis, n_model, 3, seed=n_model)
    lk = P.Likelihood("mixed")
    lk.set_T(p["T"], p["kbin"], p["n_k"], 100.0)
    lk.set_data(p["d"], p["noise_var"])
    lk.precompute()
    M = O.herm_dense(p["T"], p["noise_var"])
    db = O.dbar_dense(p["T"], p["noise_var"], p["d"])
    ph = np.random.default_rng(n_model).uniform(-1, 1, (3, 3))
    got, st = lk.lnl(ph)
    ref = np.array([O.evaluate(M, db, p["kbin"], q, 100.0)["lnl"] for q in ph])
    record(f"random {n_vis}x{n_model}", lk, np.abs(got - ref).max())
# an uneven batch (240 and 3280 modes) and a posterior mean
a, b = make_like(P, "C0", "mixed"), make_like(P, "C1", "mixed")
pa, pb = phis("C0", 3), phis("C1", 2)
outs, sts = P.lnl_multi([a, b], [pa, pb])
ref = oracle_eval("C1", pb[0])["lnl"]
record("C0 + C1 batch", b, abs(outs[1][0] - ref))
abar, st = a.posterior_mean(pa[0])
aref = oracle_eval("C0", pa[0])["abar"]
record("posterior mean C0", a, np.linalg.norm(abar - aref) / np.linalg.norm(aref))
print("RESULT " + json.dumps(out))
"""


def test_bounds_checked_build_reports_no_failed_check():
    sys.path.insert(0, ROOT)
    from paper_2501_12928_gb300 import _build
    lib = _build.build(variant="checked")
    env = dict(os.environ, BEOR_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    print(res)
    assert res["build_info"] & 1
    tol = {"C0 fp64": 1e-7, "posterior mean C0": 1e-6}
    for c in res["cases"]:
        assert c["bounds"] == 0, c
        assert c["err"] <= tol.get(c["name"], 1e-2), c
