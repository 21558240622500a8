"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package draws the random numbers and builds the instrument forward model
that the likelihood consumes as *inputs*: per-frequency visibility response
matrices A_f, the spectral basis W, the data vector d, the noise variances,
the mode-to-k-bin map and the prior amplitudes phi.  It holds none of the
likelihood arithmetic (no T^H N^-1 T, no Sigma, no factorisation, no lnL).
"""

from .instrument import (  # noqa: F401
    CONFIGS,
    Instrument,
    InstrumentSpec,
    build_instrument,
    draw_phi,
    expand_T,
    geometry,
    get_spec,
)
