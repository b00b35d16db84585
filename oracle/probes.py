"""Rademacher probe vectors from a counter-based SplitMix64 hash (test infrastructure only).

Sec. 2.2 "Stochastic Trace Estimation": Hutchinson's estimator uses random vectors
with independent +-1 (Rademacher) entries.

Generator.  SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by
the golden-ratio increment 0x9E3779B97F4A7C15 and each output is the state passed
through the finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
``mix(x)`` below is the output produced from state x.  The sign of entry
(row, col) of stream ``stream`` under seed ``seed`` is

    h = mix( mix( mix(seed) ^ stream ) ^ ((col << 32) | row) )
    eps = -1 if the top bit of h is set else +1

stream 1 gives eps1 (k x l, rows = preconditioner columns), stream 2 gives eps2
(n x l, rows = data points).

Probe distribution.  Preconditioned CG from right-hand side z is Lanczos on
P^-1/2 K_hat P^-1/2 started at P^-1/2 z, so for the quadrature to estimate
tr(log(P^-1/2 K_hat P^-1/2)) without bias the probes need E[z z^T] = P_hat.
They are drawn as  z_i = L eps1_i + sigma eps2_i  (E[z z^T] = L L^T + sigma^2 I).
With k = 0 this is sigma times a plain Rademacher vector.  The literal Alg. 1
(normalised Rademacher z = eps2 / sqrt(n)) is kept behind ``literal=True`` so the
tests can show that it is biased when P_hat is not a multiple of I.
"""
import numpy as np

_MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB


def mix_int(x):
    """SplitMix64 output from state x (Python ints, exact)."""
    z = (x + GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * M1) & _MASK
    z = ((z ^ (z >> 27)) * M2) & _MASK
    return z ^ (z >> 31)


def splitmix64_sequence(seed, count):
    """The first ``count`` outputs of a SplitMix64 generator seeded with ``seed``."""
    out, state = [], seed & _MASK
    for _ in range(count):
        out.append(mix_int(state))
        state = (state + GOLDEN) & _MASK
    return out


def _mix_array(x):
    x = x.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def stream_key(seed, stream):
    return mix_int(mix_int(seed & _MASK) ^ stream)


def rademacher(seed, stream, rows, cols):
    """rows x cols matrix of +-1.0 from the counter hash above."""
    key = np.uint64(stream_key(seed, stream))
    r = np.arange(rows, dtype=np.uint64)[:, None]
    c = np.arange(cols, dtype=np.uint64)[None, :]
    h = _mix_array(key ^ ((c << np.uint64(32)) | r))
    top = (h >> np.uint64(63)).astype(np.int64)
    return 1.0 - 2.0 * top.astype(np.float64)


def eps_pair(seed, k, n, n_probes):
    return rademacher(seed, 1, k, n_probes), rademacher(seed, 2, n, n_probes)


def probes(L, sigma2, eps1, eps2, literal=False):
    """z_i = L eps1_i + sigma eps2_i  (or eps2_i / sqrt(n) when literal)."""
    n = eps2.shape[0]
    if literal:
        return eps2 / np.sqrt(n)
    rank = L.shape[1]
    return L @ eps1[:rank] + np.sqrt(sigma2) * eps2
