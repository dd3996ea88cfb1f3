"""Pin of the oracle's Philox4x64-10 against an independent implementation:
numpy's ``Philox`` bit generator (which increments the counter before each
block), plus basic properties of the uniform and normal draws."""
import numpy as np

from oracle import oracle as O


def test_philox_matches_numpy():
    rng = np.random.default_rng(123)
    for _ in range(50):
        ctr = rng.integers(0, 2 ** 63, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64)
        bg = np.random.Philox(counter=ctr, key=key)
        ref = bg.random_raw(4)
        c1 = ctr.copy()
        c1[0] += np.uint64(1)
        assert np.array_equal(O.philox(c1, key), ref)


def test_philox_counter_carry_matches_numpy():
    ctr = np.array([2 ** 64 - 1, 7, 0, 0], dtype=np.uint64)
    key = np.array([1, 2], dtype=np.uint64)
    ref = np.random.Philox(counter=ctr, key=key).random_raw(4)
    assert np.array_equal(O.philox(np.array([0, 8, 0, 0], dtype=np.uint64), key), ref)


def test_uniform_is_open_interval_and_flat():
    assert 0.0 < O.u01(0) < 1e-15
    assert 1.0 - 1e-15 < O.u01(2 ** 64 - 1) < 1.0
    rng = np.random.default_rng(0)
    u = np.array([O.u01(int(x)) for x in rng.integers(0, 2 ** 63, 20000, dtype=np.uint64) * 2])
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.003
