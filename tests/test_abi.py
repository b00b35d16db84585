"""The C ABI library builds, loads and exports every function include/gp.h declares.

Host-side behaviour that needs no GPU is checked here too: workspace-size
queries, status strings, and argument validation (an invalid call returns
GP_ERR_INVALID_ARG and launches nothing).
"""
import ctypes

import numpy as np
import pytest

from paper_2107_00243_gb300 import build, gp


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gp.load()


def test_exports_every_declared_symbol(lib):
    names = gp.declared_functions()
    assert {"gp_pivchol", "gp_kernel_mvm", "gp_kernel_grad_mvm", "gp_mbcg",
            "gp_mll_and_grad", "gp_workspace_size"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_workspace_sizes_are_positive_and_monotone(lib):
    s1 = gp.gp_workspace_size(gp.FN_MLL_AND_GRAD, 1000, 3, 20, 11, gp.FP64, 200)
    s2 = gp.gp_workspace_size(gp.FN_MLL_AND_GRAD, 100000, 16, 200, 33, gp.FP32, 1000)
    assert 0 < s1 < s2
    for fn in range(5):
        assert gp.gp_workspace_size(fn, 777, 5, 7, 9, gp.FP32, 50) > 0
    assert gp.gp_workspace_size(99, 10, 1, 0, 1, gp.FP32, 1) == 0
    assert gp.gp_workspace_size(gp.FN_KERNEL_MVM, 10, 0, 0, 1, gp.FP32, 1) == 0


def test_status_strings(lib):
    assert lib.gp_status_string(0) == b"GP_OK"
    assert lib.gp_status_string(-3) == b"GP_ERR_NOT_SPD"
    assert lib.gp_status_string(12345) == b"GP_UNKNOWN_STATUS"


def test_invalid_arguments_rejected_on_host(lib):
    P = gp._Problem(0, 3, 0, 1, gp.FP32, 0, 0)          # n = 0
    r = lib.gp_kernel_mvm(ctypes.byref(P), None, 1, 1, None, 1, None, 0, None)
    assert r == -1 and b"n=0" in lib.gp_last_error_message()
    P = gp._Problem(10, 40, 0, 1, gp.FP32, 1, 1)        # d too large
    assert lib.gp_kernel_mvm(ctypes.byref(P), 8, 10, 1, 16, 10, None, 0, None) == -1
    P = gp._Problem(10, 3, 42, 1, gp.FP32, 1, 1)        # unknown kernel
    assert lib.gp_kernel_mvm(ctypes.byref(P), 8, 10, 1, 16, 10, None, 0, None) == -1
    P = gp._Problem(10, 3, 0, 1, gp.FP32, 1, 1)
    assert lib.gp_kernel_mvm(ctypes.byref(P), 8, 10, 1, 8, 10, None, 0, None) == -1  # W aliases V
    r = lib.gp_kernel_mvm(ctypes.byref(P), 8, 10, 1, 16, 10, None, 0, None)
    assert r == -4                                       # workspace too small
    o = gp.opts(max_iter=0)
    assert lib.gp_mll_and_grad(ctypes.byref(P), 8, 2, 3, None, None, None, 16, 32,
                               ctypes.byref(o), None, 0, None) == -1
    o = gp.opts()
    assert lib.gp_mll_and_grad(ctypes.byref(P), 8, 11, 3, None, None, None, 16, 32,
                               ctypes.byref(o), None, 0, None) == -1          # k > n
    assert lib.gp_pivchol(None, 2, 0.0, None, None, 10, None, None, None, 0, None) == -1
    assert lib.gp_rademacher(0, 3, 10, 1, 8, None) == -1
    assert lib.gp_measure_peaks(None, None, None) == -1   # rejected before any launch
    assert lib.gp_peaks_scratch_elems() >= 8 * 256


def test_batched_workspace_size_is_sum_of_aligned_slices():
    """Host-only query: one 256-byte aligned single-call workspace per problem."""
    shapes = [(300, 4, gp.BF16), (1234, 8, gp.FP32), (4000, 12, gp.BF16)]
    k, nl, mi = 20, 8, 300
    want = 0
    for n, d, prec in shapes:
        sz = gp.gp_workspace_size(gp.FN_MLL_AND_GRAD, n, d, k, nl + 1, prec, mi)
        want += (sz + 255) // 256 * 256
    arr = (gp._Problem * len(shapes))(*[gp._Problem(n, d, gp.RBF, 0, prec, 0, 0)
                                        for n, d, prec in shapes])
    lib = gp.load()
    assert lib.gp_workspace_size_batched(len(shapes), arr, k, nl, mi) == want
    assert lib.gp_workspace_size_batched(0, arr, k, nl, mi) == 0


def test_override_marshalling():
    """A pivot order shorter than k is padded with -1 (which stops the factor on the
    device), a longer one is rejected before any device call."""
    import numpy as np
    import torch
    po = gp._piv_override([3, 1], 4, "cpu")
    assert po.dtype == torch.int32 and po.tolist() == [3, 1, -1, -1]
    assert gp._piv_override(np.array([5, 0, 2]), 3, "cpu").tolist() == [5, 0, 2]
    with pytest.raises(ValueError):
        gp._piv_override([0, 1, 2, 3, 4], 4, "cpu")


@pytest.mark.parametrize("mbar,d", [(2, 1), (4, 1), (16, 1), (64, 1), (6, 2), (8, 3), (4, 5)])
def test_quadrature_rule_matches_the_oracle(lib, mbar, d):
    """The host Gauss-Hermite rule of gp_mll_and_grad_qff (Sturm bisection for the nodes,
    Christoffel numbers for the weights) against the oracle's grid (numpy's hermgauss):
    same frequencies in the same order, same weights."""
    from oracle import features
    U, W = gp.gp_qff_rule(mbar, d)
    Uo, Wo = features.hermite_grid(mbar, d)
    assert U.shape == Uo.shape and W.shape == Wo.shape
    np.testing.assert_allclose(U, Uo, rtol=0, atol=1e-12 * max(1.0, float(np.abs(Uo).max())))
    np.testing.assert_allclose(W, Wo, rtol=1e-10, atol=1e-300)
    assert lib.gp_qff_rule(5, 1, None, None) < 0          # odd mbar
    assert lib.gp_qff_rule(8, 5, None, None) < 0          # 8^5 features exceed the limit
