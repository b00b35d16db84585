"""Pins for oracle/probes.py.

* SplitMix64 reproduces the published seed-0 outputs (tests/golden).
* The vectorised numpy hash equals the exact Python-integer hash entry by entry.
* Signs are +-1, balanced, and the two streams are uncorrelated.
* Averaged over every sign pattern, z = L eps1 + sigma eps2 has covariance exactly
  P_hat = sigma^2 I + L L^T.
"""
import itertools
import os

import numpy as np

from oracle import probes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def _golden():
    with open(GOLDEN) as f:
        return [int(line, 16) for line in f if line.strip() and not line.startswith("#")]


def test_splitmix64_published_vectors():
    assert probes.splitmix64_sequence(0, 3) == _golden()


def test_vectorised_hash_matches_integer_hash():
    seed, stream = 12345, 2
    S = probes.rademacher(seed, stream, 37, 5)
    key = probes.stream_key(seed, stream)
    for r in (0, 1, 17, 36):
        for c in (0, 3, 4):
            h = probes.mix_int(key ^ ((c << 32) | r))
            assert S[r, c] == (-1.0 if h >> 63 else 1.0)


def test_signs_balanced_and_streams_independent():
    e1 = probes.rademacher(7, 1, 20000, 4)
    e2 = probes.rademacher(7, 2, 20000, 4)
    assert set(np.unique(e1)) == {-1.0, 1.0}
    assert abs(e1.mean()) < 0.02 and abs(e2.mean()) < 0.02
    assert abs(np.mean(e1 * e2)) < 0.02
    assert not np.array_equal(probes.rademacher(7, 2, 50, 1), probes.rademacher(8, 2, 50, 1))


def test_probe_covariance_is_P_by_enumeration():
    rng = np.random.default_rng(0)
    n, k, s2 = 4, 2, 0.3
    L = rng.standard_normal((n, k))
    acc = np.zeros((n, n))
    count = 0
    for bits in itertools.product([-1.0, 1.0], repeat=n + k):
        e1 = np.array(bits[:k])[:, None]
        e2 = np.array(bits[k:])[:, None]
        z = probes.probes(L, s2, e1, e2)
        acc += z @ z.T
        count += 1
    np.testing.assert_allclose(acc / count, s2 * np.eye(n) + L @ L.T, atol=1e-13)
