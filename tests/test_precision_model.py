"""The mixed-precision arithmetic of the tensor-core kernel product, emulated in numpy,
against the exact product: the element-wise bound that the GPU parity tests use follows
from the arithmetic, not from the kernel.

The emulated steps (the mixed-precision reading of the kernel product, Sec. 2.2 product
with V):
  * exponent S = -c r^2 / 2 from augmented operands A_i = [c x_i, 1, -c|x_i|^2/2],
    B_j = [x_j, -c|x_j|^2/2, 1], each split into BF16 hi + lo parts and multiplied as
    hi.hi + hi.lo + lo.hi with FP32 accumulation (c = log2 e for RBF);
  * P = 2^S rounded to FP16 (fast mode), or FP16 hi + lo (split mode);
  * each column of V scaled by 2^e_c with max |V_c| in [2^13, 2^14), split into FP16
    hi + lo; O = P V_hi + P V_lo;
  * W = s 2^-e_c O + sigma^2 V.
The exact reference is (K + sigma^2 I) V in float64.  Per element the bound is
  |W - W_exact|_i <= sum_j K_ij (e_P + ln2 dS_ij + 2^-21) |V_j| + s 2^-25 sum_j |V_j|
with
  * e_P = 2^-11 in fast mode (FP16 rounding of P), 0 in split mode;
  * dS_ij = 2^-16 c (|x_i| + |x_j|)^2 / 2: the exponent error.  The BF16 hi + lo split
    leaves 2^-18 of each operand, and dropping lo.lo adds 2^-18 more, so each product
    term is off by at most 3 * 2^-18 < 2^-16 of |A_ik| |B_jk|.  By Cauchy-Schwarz the
    sum over k of those products is at most c (|x_i| + |x_j|)^2 / 2;
  * 2^-21 for the FP16 hi + lo residue of the scaled V and of P in split mode;
  * s 2^-25 for values of P in FP16's subnormal range (absolute rounding).
In split mode P carries 22 bits, so the exponent's ~16 bits set the error there.  Fast
mode also stays within the 2^-10 (|K| |V|)_i that the GPU parity tests use.
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


def _split_bf16(a):
    hi = _bf16(a)
    lo = _bf16(np.asarray(a, np.float32) - hi)
    return hi, lo


def _emulated_product(X, s, s2, V, split):
    c = L2E
    nrm = (X.astype(np.float64) ** 2).sum(1)
    A = np.concatenate([c * X, np.ones((len(X), 1)), -c * nrm[:, None] / 2], 1).astype(np.float32)
    B = np.concatenate([X, -c * nrm[:, None] / 2, np.ones((len(X), 1))], 1).astype(np.float32)
    Ah, Al = _split_bf16(A)
    Bh, Bl = _split_bf16(B)
    f64 = np.float64
    S = (Ah.astype(f64) @ Bh.T.astype(f64) + Ah.astype(f64) @ Bl.T.astype(f64)
         + Al.astype(f64) @ Bh.T.astype(f64)).astype(np.float32)
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
    dS = 2.0 ** -16 * L2E * (nx[:, None] + nx[None, :]) ** 2 / 2
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
