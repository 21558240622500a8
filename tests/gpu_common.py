"""Helpers shared by the GPU parity tests (inputs and oracle references)."""

import functools

import numpy as np

import oracle as O
from synth import build_instrument, draw_phi, expand_T
from synth.instrument import get_spec


@functools.lru_cache(maxsize=None)
def instrument(name, **over):
    spec = get_spec(name.split(":")[0], **dict(over)) if over else name
    return build_instrument(spec)


@functools.lru_cache(maxsize=None)
def oracle_pre(name, dense=False):
    inst = instrument(name)
    if dense:
        T = expand_T(inst)
        return O.herm_dense(T, inst.noise_var), O.dbar_dense(T, inst.noise_var, inst.d)
    return (O.herm_structured(inst.A, inst.W, inst.noise_var),
            O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d))


def oracle_eval(name, phi):
    inst = instrument(name)
    M, db = oracle_pre(name)
    return O.evaluate(M, db, inst.kbin, phi, inst.spec.lssm_prior_var)


def make_like(P, name, precision="fp64", dense=False):
    inst = instrument(name)
    lk = P.Likelihood(precision)
    if dense:
        lk.set_T(expand_T(inst), inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    else:
        lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    lk.precompute()
    return lk


def phis(name, n, stream=3):
    return draw_phi(instrument(name).spec, n, stream=stream)
