"""The seeded NFIR input generator (shared input data, no GP arithmetic)."""
import numpy as np

import nfir


def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014) from seed 0: its first outputs as published with the
    reference implementation."""
    z = nfir.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_dataset_shapes_lags_and_determinism():
    X, y, Xs, ys = nfir.make_dataset(500, 100, 8, 0)
    assert X.shape == (500, 8) and y.shape == (500,) and Xs.shape == (100, 8) and ys.shape == (100,)
    assert np.array_equal(X[1:, 1:], X[:-1, :-1])  # column d is the force lagged by d samples
    X2, y2, _, _ = nfir.make_dataset(500, 100, 8, 0)
    assert np.array_equal(X, X2) and np.array_equal(y, y2)
    X3, *_ = nfir.make_dataset(500, 100, 8, 1)
    assert not np.array_equal(X, X3)
    assert np.all(np.abs(X) <= 1.0)


def test_force_is_held_for_twenty_samples():
    u, y = nfir.simulate(400, 5)
    blocks = u.reshape(20, 20)
    assert np.all(blocks == blocks[:, :1])
    assert len(np.unique(u)) == 20


def test_batch_sizes_in_range():
    ns, Ds = nfir.batch_sizes(512)
    assert ns.min() >= 128 and ns.max() <= 4096 and set(Ds.tolist()) <= {4, 8, 16}
