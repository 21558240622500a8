"""Host-side batching of the exact likelihood used by the samplers: batches
are padded to powers of two (so the library keeps one captured graph and
one set of workspaces per size, at most log2(max_batch) + 1 of them),
padding rows are neither returned nor counted, a point whose status is a
failed pivot (or a non-finite phi) gets lnL = -inf, a point flagged as
possibly outside the mixed-precision tolerance is re-evaluated on the
float64 fallback or rejected, and record mode keeps every evaluated pair."""

import numpy as np

from paper_2501_12928_gb300.emulated_sampler import ExactLikelihood


class FakeLike:
    """Stands in for the library: lnL = -sum(phi^2), status 7 where phi[0] > 1.5."""

    def __init__(self):
        self.sizes = []

    def lnl(self, phi):
        phi = np.asarray(phi)
        self.sizes.append(len(phi))
        st = np.where(phi[:, 0] > 1.5, 7, 0).astype(np.int32)
        return -np.sum(phi ** 2, axis=1), st


def test_power_of_two_batches_and_padding():
    fake = FakeLike()
    ex = ExactLikelihood(fake, max_batch=64)
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 63, 64, 65, 200):
        x = rng.uniform(-2, 2, (n, 9))
        x[:, 0] = np.clip(x[:, 0], -2, 1.4)
        got = ex(x)
        assert got.shape == (n,)
        np.testing.assert_array_equal(got, -np.sum(x ** 2, axis=1))
    assert all(s & (s - 1) == 0 and s <= 64 for s in fake.sizes), fake.sizes
    assert len(set(fake.sizes)) <= int(np.log2(64)) + 1
    assert ex.n_points == 1 + 2 + 3 + 63 + 64 + 65 + 200


def test_failed_points_are_minus_infinity_and_recorded():
    ex = ExactLikelihood(FakeLike(), max_batch=8)
    ex.record = True
    x = np.zeros((5, 3))
    x[2, 0] = 1.9
    got = ex(x)
    assert got[2] == -np.inf and np.all(np.isfinite(np.delete(got, 2)))
    assert len(ex.rec_x) == 1 and ex.rec_x[0].shape == (5, 3)
    np.testing.assert_array_equal(ex.rec_l[0], got)


class FlagLike:
    """Stands in for the mixed-precision library: lnL = -sum(phi^2) + 0.5 (an
    error the tolerance estimate caught), status -1 where phi[1] > 1, status
    -2 where phi[2] > 1.9."""

    def __init__(self):
        self.calls = 0

    def lnl(self, phi):
        phi = np.asarray(phi)
        self.calls += 1
        st = np.where(phi[:, 1] > 1.0, -1, 0).astype(np.int32)
        st = np.where(phi[:, 2] > 1.9, -2, st).astype(np.int32)
        return -np.sum(phi ** 2, axis=1) + 0.5, st


class F64Like:
    """Stands in for the float64 fallback: the exact lnL = -sum(phi^2)."""

    def __init__(self):
        self.sizes = []

    def lnl(self, phi):
        phi = np.asarray(phi)
        self.sizes.append(len(phi))
        return -np.sum(phi ** 2, axis=1), np.zeros(len(phi), np.int32)


def _points():
    x = np.zeros((7, 3))
    x[1, 1] = 1.5       # flagged
    x[4, 1] = 1.2       # flagged
    x[5, 2] = 1.95      # non-finite phi stand-in (status -2)
    return x


def test_flagged_points_use_the_float64_fallback():
    fb = F64Like()
    ex = ExactLikelihood(FlagLike(), max_batch=4, fallback=fb)
    x = _points()
    got = ex(x)
    exact = -np.sum(x ** 2, axis=1)
    for b in (1, 4):
        assert got[b] == exact[b]                     # the fallback's value, not the flagged one
    assert got[5] == -np.inf
    for b in (0, 2, 3, 6):
        assert got[b] == exact[b] + 0.5               # unflagged mixed results pass through
    assert ex.n_flagged == 2 and ex.n_fallback == 2
    assert all(s & (s - 1) == 0 for s in fb.sizes)    # fallback batches are powers of two too


def test_flagged_points_are_rejected_without_fallback():
    ex = ExactLikelihood(FlagLike(), max_batch=8)
    ex.record = True
    got = ex(_points())
    assert got[1] == -np.inf and got[4] == -np.inf and got[5] == -np.inf
    assert ex.n_flagged == 2 and ex.n_fallback == 0
    np.testing.assert_array_equal(ex.rec_l[0], got)   # the training record never holds a flagged value
