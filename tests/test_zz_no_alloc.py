"""The allocation-free dbar entry point against the regular precompute.

beor_dbar_factored_noalloc serves callers that cannot allocate device memory
(their framework owns all of it, or they must not stall on the allocator):
it computes dbar = T^H N^-1 d of a factored instrument with its scratch in a
fixed device array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _instrument():
    from synth import build_instrument
    from synth.instrument import get_spec
    return build_instrument(get_spec("C1", nu=5, nf=6, n_t=3, n_bl=20, n_pix=16, n_k=3))


def test_noalloc_dbar_matches_precompute_twice():
    import torch

    import paper_2501_12928_gb300 as P
    from paper_2501_12928_gb300 import beor as B

    inst = _instrument()
    lk = P.Likelihood("fp64")
    lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    lk.precompute()
    ref = lk.get_dbar()

    nf, ntb, nc = inst.A.shape
    nx = inst.W.shape[1]
    dev = torch.device("cuda")
    A = torch.from_numpy(np.ascontiguousarray(inst.A)).to(dev)
    W = torch.from_numpy(np.ascontiguousarray(inst.W)).to(dev)
    nv = torch.from_numpy(np.ascontiguousarray(inst.noise_var)).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(inst.d)).to(dev)
    lib = B._lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):   # two calls in a row share the scratch array
        out = torch.full((nc * nx,), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
        rc = lib.beor_dbar_factored_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(W.data_ptr()), nf, ntb,
                                            nc, nx, ctypes.c_void_p(nv.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.beor_strerror(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()

    # sizes beyond the fixed scratch are rejected, and host pointers too
    rc = lib.beor_dbar_factored_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(W.data_ptr()), 65537, ntb,
                                        1, nx, ctypes.c_void_p(nv.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == -1
    host = np.zeros(nc * nx, np.complex128)
    rc = lib.beor_dbar_factored_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(W.data_ptr()), nf, ntb, nc,
                                        nx, ctypes.c_void_p(nv.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                        ctypes.c_void_p(host.ctypes.data), stream)
    assert rc == -1
