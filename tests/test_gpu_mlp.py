"""Emulator network kernels (bf16 tensor-core GEMMs, fp32 accumulation) against
the float64 oracle: gradients within bf16 bounds (cosine >= 0.999, relative
L2 <= 2e-2), forward outputs, and training that reduces the loss."""

import numpy as np
import pytest

from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2501_12928_gb300 as P
    return P


def _bf16(a):
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16       # round to nearest even
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(em, bf16=True):
    out = []
    for l in range(em.depth + 1):
        W, b = em.get_params(l)
        out.append((_bf16(W) if bf16 else W.astype(np.float64), b.astype(np.float64)))
    return out


def _data(n, seed=0):
    g = np.random.default_rng(seed)
    x = g.uniform(-2, 2, (n, 9)).astype(np.float32)
    t = (50.0 - 3.0 * np.sum((x - 0.3) ** 2, axis=1) + 2.0 * x[:, 0] * x[:, 1]).astype(np.float32)
    return x, t


NORM = (np.zeros(9, np.float32), np.full(9, 0.5, np.float32), 40.0, 20.0)


def test_gradients_match_oracle(P):
    em = P.Emulator(9, 256, 4, seed=4)
    em.set_norm(*NORM)
    x, t = _data(512)
    params = _params(em)
    loss_ref, grads_ref = OM.loss_and_grads(params, x.astype(np.float64), t.astype(np.float64),
                                            NORM[0].astype(np.float64), NORM[1].astype(np.float64), NORM[2], NORM[3])
    for l in range(em.depth + 1):
        dW, db, loss = em.grad(x, t, l)
        gr = grads_ref[l][0]
        cos = float(np.sum(dW * gr) / (np.linalg.norm(dW) * np.linalg.norm(gr)))
        rel = float(np.linalg.norm(dW - gr) / np.linalg.norm(gr))
        assert cos >= 0.999 and rel <= 2e-2, (l, cos, rel)
        relb = float(np.linalg.norm(db - grads_ref[l][1]) / np.linalg.norm(grads_ref[l][1]))
        assert relb <= 2e-2, (l, relb)
        assert abs(loss - loss_ref) <= 2e-2 * loss_ref


def test_forward_matches_oracle(P):
    em = P.Emulator(9, 256, 4, seed=7)
    em.set_norm(*NORM)
    x, _ = _data(3000, seed=1)
    y = em.infer(x)
    ref, _ = OM.forward(_params(em), x.astype(np.float64), NORM[0], NORM[1])
    ref = ref * NORM[3] + NORM[2]
    assert np.linalg.norm(y - ref) <= 2e-2 * np.linalg.norm(ref - ref.mean()) + 1e-3 * np.linalg.norm(ref)


def test_training_reduces_loss(P):
    em = P.Emulator(9, 256, 4, seed=4)
    em.set_norm(*NORM)
    x, t = _data(8192, seed=2)
    first = None
    for epoch in range(30):
        perm = np.random.default_rng(epoch).permutation(len(x))
        for i in range(0, len(x), 1024):
            sel = perm[i:i + 1024]
            loss = em.train_step(x[sel], t[sel], 1e-3)
            if first is None:
                first = loss
    xv, tv = _data(2000, seed=3)
    pred = em.infer(xv)
    rms = float(np.sqrt(np.mean((pred - tv) ** 2)))
    assert loss < 0.05 * first, (first, loss)
    assert rms < 0.1 * float(np.std(tv)), rms
