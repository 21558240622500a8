"""The tensor-core precompute of M = T^H N^-1 T from a dense T (mixed
contexts: seven-digit bf16 slice products over K-blocks of 128
visibilities, double-float accumulation across blocks) against the oracle:
the dense float64 product on the 240-mode instrument, the independent
structured form on the 3280-mode instrument (90,972 visibilities), and lnL
on the mixed path.  Also reports the dense precompute's time on the tensor
cores and on the float64 path.

Bound on M: the operands carry 56 bits and levels 0-2 are exact, but the
fourth level's fp32 accumulator (pairs s + t >= 3, 2^-24 below the leading
term) rounds once per product it receives, about 320 times per K-block, and
the roundings add up almost linearly: up to about 2^-48 x 320 ~ 2^-40 of
the largest element per block.  The bound 2^-38 of max |M| is below
float64 accumulation's own worst case over these K (K 2^-53, 1e-11 at
90,972 visibilities); lnL parity is the criterion that matters."""

import time

import numpy as np
import pytest

import oracle as O
from gpu_common import instrument, oracle_pre, phis

pytestmark = pytest.mark.gpu


def _dense_like(P, inst, precision, T):
    lk = P.Likelihood(precision)
    lk.set_T(T, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lk.precompute()
    return lk, time.perf_counter() - t0


def test_tensor_core_precompute_C0():
    import paper_2501_12928_gb300 as P
    from synth import expand_T

    inst = instrument("C0")
    T = expand_T(inst)
    lk, _ = _dense_like(P, inst, "mixed", T)
    M_ref = O.herm_dense(T, inst.noise_var)
    M = lk.get_M()
    err = np.abs(M - M_ref).max() / np.abs(M_ref).max()
    print("C0 tensor-core M relative error", err)
    assert err <= 2.0 ** -38
    assert np.all(M.diagonal().imag == 0.0)
    np.testing.assert_array_equal(M, M.conj().T)
    ph = phis("C0", 8)
    got, st = lk.lnl(ph)
    assert np.all(st == 0)
    Ms, dbs = oracle_pre("C0")
    ref = np.array([O.evaluate(Ms, dbs, inst.kbin, p, inst.spec.lssm_prior_var)["lnl"] for p in ph])
    assert np.abs(got - ref).max() <= 1e-2
    lk.close()


@pytest.mark.slow
def test_tensor_core_precompute_C1_dense():
    import paper_2501_12928_gb300 as P
    from synth import expand_T

    inst = instrument("C1")
    T = expand_T(inst)                      # 90,972 x 3280 complex128 (4.8 GB)
    lk, t_tc = _dense_like(P, inst, "mixed", T)
    _, t_tc2 = _dense_like(P, inst, "mixed", T)   # second run: no first-use costs
    lf, t_f64 = _dense_like(P, inst, "fp64", T)
    print(f"dense precompute at N_model 3280, n_vis 90972: tensor cores {t_tc2:.3f} s "
          f"(first call {t_tc:.3f} s), float64 pipe {t_f64:.3f} s")
    M_ref, db_ref = oracle_pre("C1")        # structured form: never forms T
    M = lk.get_M()
    err = np.abs(M - M_ref).max() / np.abs(M_ref).max()
    err64 = np.abs(lf.get_M() - M_ref).max() / np.abs(M_ref).max()
    print("C1 M relative error: tensor cores", err, "float64 pipe", err64)
    assert err <= 2.0 ** -38
    ph = phis("C1", 2)
    got, st = lk.lnl(ph)
    assert np.all(st == 0)
    for b in range(2):
        ref = O.evaluate(M_ref, db_ref, inst.kbin, ph[b], inst.spec.lssm_prior_var)["lnl"]
        print("C1 dense mixed |dlnL|", abs(got[b] - ref))
        assert abs(got[b] - ref) <= 1e-2
    lk.close()
    lf.close()
