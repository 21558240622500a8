"""CPU float64 oracle for the BayesEoR likelihood hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library (no kernels, headers, helpers, tables or pre/post-processing)
and never imports it.  It is plain, slow and written to be checked by eye
against the definitions it cites.

Parity status: every function here is pinned by the tests in
``tests/test_oracle_pins.py`` (brute-force Woodbury / determinant-lemma
evaluation, the unitary-T closed form, dense-vs-structured precompute,
library Cholesky/slogdet, posterior-mean limits, finite-difference
derivatives, MLP finite differences).  The one exception is the realism of
the synthetic workloads themselves, which the paper gives no values for
(parity unpinned against the paper's test dataset).
"""

from .likelihood import (  # noqa: F401
    cholesky_lower,
    dbar_dense,
    dbar_structured,
    evaluate,
    forward_sub,
    back_sub,
    herm_dense,
    herm_structured,
    prior_diag,
)
