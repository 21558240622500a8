"""Writes tests/golden/c0_oracle.json: oracle lnL values on the 240-mode workload.

Calls only the oracle (and the seeded input generator).  Re-run with
`python tests/golden/make_golden.py` after a justified change of the oracle.
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from synth import build_instrument, draw_phi  # noqa: E402


def main():
    inst = build_instrument("C0")
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    phis = draw_phi("C0", 16)
    rows = []
    for phi in phis:
        r = O.evaluate(M, db, inst.kbin, phi, inst.spec.lssm_prior_var)
        rows.append({"phi": [float(x) for x in phi], "lnl": r["lnl"],
                     "logdet_phi": r["logdet_phi"], "logdet_sigma": r["logdet_sigma"], "q": r["q"]})
    out = {"source": "oracle.likelihood.evaluate on synth C0 (seeded); phi = draw_phi('C0', 16)",
           "n_model": inst.n_model, "n_vis": inst.n_vis, "rows": rows}
    with open(os.path.join(HERE, "c0_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
