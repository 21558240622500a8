"""GB300-native exact likelihood of the BayesEoR 21-cm power-spectrum model.

The compute runs in the CUDA library ``_build/libbeor.so`` (C ABI declared in
``include/beor.h``); this package only marshals arguments to it.
"""

from .beor import (  # noqa: F401
    BeorError,
    Likelihood,
    Emulator,
    lib,
    lnl_multi,
    lnl_multi_async,
    lnl_multi_wait,
    PREC_FP64,
    PREC_MIXED,
    KERNEL_CLASSES,
    set_lookahead,
    set_profiling,
    set_wait_test,
    set_schedule,
    get_schedule,
    autotune,
)
