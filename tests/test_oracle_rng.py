"""Pin of oracle.rng against numpy.random.Philox (an independent Philox4x64-10)."""
import numpy as np

from oracle import rng


def test_philox_matches_numpy_bitgenerator():
    # numpy's generator advances the counter before each 4-word block
    for key, ctr in (((0, 0), (0, 0, 0, 0)), ((5, 7), (10, 20, 30, 40)),
                     ((2**64 - 1, 123456789), (2**64 - 3, 2**64 - 1, 7, 9))):
        g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
        ref = g.random_raw(12)
        c = list(ctr)
        for blk in range(3):
            for w in range(4):             # 256-bit increment with carry
                c[w] = (c[w] + 1) % 2**64
                if c[w] != 0:
                    break
            out = rng.philox4x64(*[np.uint64(v) for v in c], np.uint64(key[0]), np.uint64(key[1]))
            assert [int(o) for o in out] == [int(v) for v in ref[4 * blk:4 * blk + 4]]


def test_uniform_open_interval_and_exact():
    x = np.array([0, 2**64 - 1, 2**63, 4095, 4096], dtype=np.uint64)
    u = rng.uniform(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 0.5 * 2.0**-52 and u[1] == 1.0 - 0.5 * 2.0**-52
    assert u[4] == 1.5 * 2.0**-52


def test_vectorised_counters_match_scalar_calls():
    m = np.arange(5, dtype=np.uint64)
    v = rng.philox4x64(m, 3, 0, 0, 99, rng.stream_key(2, 1, 4, 17))
    for i in range(5):
        s = rng.philox4x64(np.uint64(i), 3, 0, 0, 99, rng.stream_key(2, 1, 4, 17))
        assert all(int(a[i]) == int(b) for a, b in zip(v, s))
