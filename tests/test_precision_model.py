"""The mixed-precision arithmetic of the tensor-core kernel product, emulated in numpy,
against the exact product: the element-wise bound that the GPU parity tests use follows
from the arithmetic, not from the kernel.

The emulated steps (the mixed-precision reading of the kernel product, Sec. 2.2 product
with V):
  * exponent S = -c r^2 / 2 from augmented operands A_i = [c x_i, 1, -c|x_i|^2/2],
    B_j = [x_j, -c|x_j|^2/2, 1] (c = log2 e for RBF), each entry split into BF16 parts
    v = p0 + p1 (+ p2), p_m = bf16(v - p_0 - .. - p_{m-1}), and multiplied as the
    products of total order <= 1 (fast mode: p0.q0 + p0.q1 + p1.q0) or <= 2 (split mode,
    three parts: those plus p0.q2 + p1.q1 + p2.q0).  The tensor core accumulates in
    FP32: the emulation rounds the accumulator to FP32 after every K = 16 step;
  * P = 2^S rounded to FP16 (fast mode), or FP16 hi + lo (split mode);
  * each column of V scaled by 2^e_c with max |V_c| in [2^13, 2^14), split into FP16
    hi + lo; O = P V_hi + P V_lo;
  * W = s 2^-e_c O + sigma^2 V.
The exact reference is (K + sigma^2 I) V in float64.  Per element the bound is
  |W - W_exact|_i <= sum_j K_ij (e_P + ln2 dS_ij + 2^-21) |V_j| + s 2^-25 sum_j |V_j|
with
  * e_P = 2^-11 in fast mode (FP16 rounding of P), 0 in split mode;
  * dS_ij = e_S c (|x_i| + |x_j|)^2 / 2, the exponent error.  By Cauchy-Schwarz the sum
    over k of |A_ik| |B_jk| is at most c (|x_i| + |x_j|)^2 / 2.  Fast mode: the BF16
    hi + lo split leaves 2^-18 of each operand and dropping lo.lo adds 2^-18 more, so each
    product term is off by at most 3 * 2^-18 of |A_ik| |B_jk|; with the FP32 roundings
    of the accumulator e_S = 2^-16.  Split mode: three parts leave 2^-27 of each operand
    and the dropped products of order 3 and 4 are below 3 * 2^-27, so the roundings of
    the FP32 accumulator (at most 13 K steps, 2^-24 each of a partial sum bounded by the
    same Cauchy-Schwarz sum) dominate: e_S = 2^-20;
  * 2^-21 for the FP16 hi + lo residue of the scaled V and of P in split mode;
  * s 2^-25 for values of P in FP16's subnormal range (absolute rounding).
Fast mode also stays within the 2^-10 (|K| |V|)_i that the GPU parity tests use.  On
inputs with large norms (|x|^2 ~ 30, like the n = 5e5 Gaussian-mixture workload) the
two-part exponent's error is ~2^-16 c |x|^2 ~ 7e-4 in S: the reason split mode uses
three parts.
"""
import numpy as np
import pytest

L2E = 1.4426950408889634


def _bf16(a):
    """Round float32 values to BF16 (nearest even), returned as float32."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _bf16_parts(a, parts):
    """BF16 parts p0 + p1 (+ p2) of float64 values (each part rounded from float32)."""
    a = np.asarray(a, np.float64)
    out, r = [], a.copy()
    for _ in range(parts):
        p = _bf16(r.astype(np.float32)).astype(np.float64)
        out.append(p)
        r = r - p
    return out


def _exponent(X, split):
    """S as the tensor core forms it: the kept part products, concatenated along K,
    accumulated in FP32 over K steps of 16."""
    c = L2E
    nrm = (X.astype(np.float64) ** 2).sum(1)
    A = np.concatenate([c * X, np.ones((len(X), 1)), -c * nrm[:, None] / 2], 1)
    B = np.concatenate([X, -c * nrm[:, None] / 2, np.ones((len(X), 1))], 1)
    if split:
        pa, pb = _bf16_parts(A, 3), _bf16_parts(B, 3)
        pairs = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]
    else:
        pa, pb = _bf16_parts(A, 2), _bf16_parts(B, 2)
        pairs = [(0, 0), (0, 1), (1, 0)]
    Ak = np.concatenate([pa[i] for i, _ in pairs], 1)
    Bk = np.concatenate([pb[j] for _, j in pairs], 1)
    acc = np.zeros((len(X), len(X)), np.float32)
    for k0 in range(0, Ak.shape[1], 16):
        acc = (acc.astype(np.float64) + Ak[:, k0:k0 + 16] @ Bk[:, k0:k0 + 16].T).astype(np.float32)
    return acc


def _emulated_product(X, s, s2, V, split):
    S = _exponent(X, split)
    f64 = np.float64
    Pf = np.exp2(S.astype(np.float64)).astype(np.float32)
    Ph = Pf.astype(np.float16)
    P = Ph.astype(f64)
    if split:
        P = P + (Pf - Ph.astype(np.float32)).astype(np.float16).astype(f64)
    mx = np.abs(V).max(0)
    e = 13 - np.floor(np.log2(np.where(mx > 0, mx, 1.0)))
    Vs = (V * np.exp2(e)).astype(np.float32)
    Vh = Vs.astype(np.float16)
    Vl = (Vs - Vh.astype(np.float32)).astype(np.float16)
    O = P @ Vh.astype(f64) + P @ Vl.astype(f64)
    return s * np.exp2(-e) * O + s2 * V


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("d,ls", [(16, 0.6), (4, 0.3), (2, 2.0)])
def test_mixed_product_within_derived_bound(split, d, ls):
    rng = np.random.default_rng(d)
    n, t = 600, 5
    X = (rng.uniform(0, 1, (n, d)) - 0.5) / ls            # centred, lengthscale-scaled
    s, s2 = 1.3, 0.01
    V = rng.standard_normal((n, t))
    V[:, 1] *= 1e-6                                         # columns of very different scale
    V[:, 2] = np.abs(V[:, 2])                               # one-signed column
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    K = s * np.exp(-0.5 * D2)
    W_ex = K @ V + s2 * V
    W = _emulated_product(X.astype(np.float32), s, s2, V, split)
    err = np.abs(W - W_ex)
    nx = np.sqrt((X ** 2).sum(1))
    dS = (2.0 ** -20 if split else 2.0 ** -16) * L2E * (nx[:, None] + nx[None, :]) ** 2 / 2
    rel = (0.0 if split else 2.0 ** -11) + np.log(2.0) * dS + 2.0 ** -21
    bound = (K * rel) @ np.abs(V) + s * 2.0 ** -25 * np.abs(V).sum(0)
    assert np.all(err <= bound), float(np.max(err / bound))
    scale = np.abs(K) @ np.abs(V)
    if not split:
        assert np.all(err <= 2.0 ** -10 * scale)            # the GPU tests' tolerance
        assert np.max(err / scale) > 2.0 ** -16             # FP16 rounding is visible


def test_bf16_rounding_helper():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to even (1); 1 + 3 * 2^-9 rounds up
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5], dtype=np.float32)
    assert list(_bf16(a)) == [1.0, 1.0, 1.0 + 2 ** -7, -2.5]


@pytest.mark.parametrize("split,e_s", [(False, 2.0 ** -16), (True, 2.0 ** -20)])
def test_exponent_error_bound_on_large_norm_inputs(split, e_s):
    """Inputs like the n = 5e5 workload's (a Gaussian mixture spanning [-2.5, 2.5]^10,
    |x|^2 up to ~30): the exponent stays within e_S c (|x_i| + |x_j|)^2 / 2, and the
    three-part form is more than 20x closer than the two-part one (2.7e-4 against 8.4e-6
    here; the FP32 accumulator, whose unit in the last place at |S| ~ 45 is 4e-6, is
    what limits the three-part form)."""
    rng = np.random.default_rng(5)
    means = rng.uniform(-2.0, 2.0, (20, 10))
    X = means[rng.integers(0, 20, 400)] + 0.3 * rng.standard_normal((400, 10))
    X = X - X.mean(0)
    S = _exponent(X.astype(np.float32), split).astype(np.float64)
    Xd = X.astype(np.float32).astype(np.float64)
    S_ex = -0.5 * L2E * ((Xd[:, None, :] - Xd[None, :, :]) ** 2).sum(-1)
    nx = np.sqrt((Xd ** 2).sum(1))
    bound = e_s * L2E * (nx[:, None] + nx[None, :]) ** 2 / 2
    err = np.abs(S - S_ex)
    assert np.all(err <= bound), float(np.max(err / bound))
    if split:
        two = np.abs(_exponent(X.astype(np.float32), False).astype(np.float64) - S_ex)
        assert two.max() > 20 * err.max(), (two.max(), err.max())
