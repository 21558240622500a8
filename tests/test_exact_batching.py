"""Host-side batching of the exact likelihood used by the samplers: batches
are padded to powers of two (so the library keeps one captured graph and
one set of workspaces per size, at most log2(max_batch) + 1 of them),
padding rows are neither returned nor counted, a point whose status is a
failed pivot gets lnL = -inf, and record mode keeps every evaluated pair."""

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
