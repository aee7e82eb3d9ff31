"""The tensor-core tile GEMM (tcgen05, split precision, complex as real 2 x 2 blocks)
against an FP64 product, through the C ABI.

Bound: |Y - Z Mt^T| <= 4e-6 * (|Z| |Mt|^T) elementwise.  3xTF32 keeps each operand to
2^-22 (hi + lo, the lo part truncated to TF32) and drops only the lo*lo product (2^-22),
about 5e-7 of each product; BF16X3 keeps 3 x 8 bits (2^-24) and drops the products of
order 2^-24 and below.  FP32 accumulation over K <= 2 x 160 real terms adds at most
a few 1e-6 in the worst case.  A single TF32 or BF16 product (5e-4 / 4e-3 relative),
a dropped cross term, a wrong operand layout or a wrong sign in the 2 x 2 blocks all
fail this bound by orders of magnitude.

Drift: the tensor core rounds its FP32 accumulation toward zero (about -0.4 ulp per MMA
instruction, measured on GB300), so one accumulator carried over K = 1024 complex
(768 instructions) shrinks a sum of positive products by 1.7e-5.  The tile gives every MMA
K step its own accumulator and sums the steps in round-to-nearest: the mean signed error
over positive data must stay below 1e-7 (one full-scale truncation per step, unbiased
summation).
"""
import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("M,K,N", [(128, 32, 8), (300, 100, 40), (5, 7, 3), (1000, 160, 64), (129, 33, 20)])
def test_tc_gemm_matches_fp64(kind, M, K, N):
    rng = np.random.default_rng(M * 1000 + K * 10 + N + kind)
    Z = crandn(rng, M, K)
    Mt = crandn(rng, N, K)
    Y, st = ttns.selftest_tc_gemm(kind, Z, Mt)
    assert st == 0
    ref = Z @ Mt.T
    scale = np.abs(Z) @ np.abs(Mt).T
    err = np.abs(Y - ref) / scale
    assert err.max() < 4e-6, f"max relative error {err.max():.2e}"


def test_tc_gemm_scales_and_signs():
    # widely different magnitudes within a row and purely imaginary / real operands: the
    # split keeps the small entries' own relative accuracy only up to the row's scale
    rng = np.random.default_rng(3)
    Z = crandn(rng, 64, 40) * np.logspace(-6, 0, 40)[None, :]
    Mt = 1j * rng.standard_normal((16, 40))
    for kind in (1, 2):
        Y, st = ttns.selftest_tc_gemm(kind, Z, Mt)
        assert st == 0
        ref = Z @ Mt.T
        scale = np.abs(Z) @ np.abs(Mt).T
        assert (np.abs(Y - ref) / scale).max() < 4e-6


@pytest.mark.parametrize("kind", [1, 2])
def test_tc_gemm_has_no_accumulation_drift(kind):
    rng = np.random.default_rng(11 + kind)
    for K in (64, 1024):
        Z = rng.uniform(0.5, 1.0, (256, K)) + 0j
        Mt = rng.uniform(0.5, 1.0, (16, K)) + 0j
        Y, st = ttns.selftest_tc_gemm(kind, Z, Mt)
        assert st == 0
        ref = (Z @ Mt.T).real
        rel = (Y.real - ref) / ref
        assert abs(rel.mean()) < 1e-7, f"K={K}: mean signed error {rel.mean():.2e}"
        assert np.abs(rel).max() < 1e-6, f"K={K}: max error {np.abs(rel).max():.2e}"
