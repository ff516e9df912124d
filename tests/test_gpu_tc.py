"""The tensor-core product path (digit-split BF16 products with exact FP32
accumulation, three real products per complex one) through the C ABI's
hopf_tc_zgemm, against numpy's complex128 matrix product.

Exactness: operands whose every component (re, im, re + im) is an integer
below 128 are represented exactly by one digit, and every partial sum stays
an integer below 2^24, so the result must equal the exact product bit for
bit, across K-chunks and tile edges.  Accuracy: with S digits the error is
at most about S 2^(-8S) of (|op(A)| |op(B)|) entry by entry, also when row
and column magnitudes span sixteen orders (per-row scaling)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2403_04946_gb300 import binding, build
    build.build()
    c = binding.Context(d=4, n=8, nu=0.01, tol=1e-10, rank_cap=4, L=3.0, precision=binding.HOPF_MIXED)
    yield c
    c.close()


def op(X, o):
    return X.conj().T if o else X


def operands(rng, M, N, K, opA, opB, integer=False, graded=False):
    def mat(r, c):
        if integer:
            return (rng.integers(-63, 64, (r, c)) + 1j * rng.integers(-63, 64, (r, c))).astype(np.complex128)
        return rng.standard_normal((r, c)) + 1j * rng.standard_normal((r, c))
    A = mat(K, M) if opA else mat(M, K)
    B = mat(N, K) if opB else mat(K, N)
    if graded:  # rows of op(A) and columns of op(B) over 16 orders of magnitude
        ra = 10.0 ** rng.uniform(-8, 8, M)
        cb = 10.0 ** rng.uniform(-8, 8, N)
        A = (ra[None, :] * A) if opA else (ra[:, None] * A)
        B = (cb[:, None] * B) if opB else (B * cb[None, :])
    return A, B


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 40, 1000), (128, 32, 192), (129, 33, 193), (300, 70, 64)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_one_digit_integer_products_are_exact(ctx, M, N, K, opA, opB):
    rng = np.random.default_rng(M * 7 + N * 3 + K + 11 * opA + 13 * opB)
    A, B = operands(rng, M, N, K, opA, opB, integer=True)
    got = ctx.hopf_tc_zgemm(A, B, opA, opB, digits=1)
    np.testing.assert_array_equal(got, op(A, opA) @ op(B, opB))


@pytest.mark.parametrize("digits", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("M,N,K,opA,opB", [(200, 50, 777, 1, 0), (129, 31, 5000, 0, 1), (64, 96, 63, 0, 0)])
def test_error_falls_eight_bits_per_digit(ctx, digits, M, N, K, opA, opB):
    rng = np.random.default_rng(100 * digits + K)
    A, B = operands(rng, M, N, K, opA, opB, graded=True)
    oa, ob = op(A, opA), op(B, opB)
    want = oa @ ob
    scale = np.abs(oa) @ np.abs(ob)  # |op(A)| |op(B)|, the natural size of each entry's error
    got = ctx.hopf_tc_zgemm(A, B, opA, opB, digits=digits)
    rel = float(np.max(np.abs(got - want) / scale))
    print(f"\ndigits {digits}, {M}x{N}x{K}: max error / (|A||B|) {rel:.2e}")
    assert rel <= 2.0 ** (-8 * digits + 5)  # 5 digits: 2.9e-11


@pytest.mark.parametrize("digits", [2, 3, 5])
def test_values_just_below_a_power_of_two(ctx, digits):
    """Entries within 2^-32 .. 2^-50 below a power of two (and their
    negatives): the row scale puts them at the top of the digit range, where
    the integer carried into the next digit is largest (a value like
    Phi(a) = 1 - 1e-12 near a = 0).  Same error bound as random data."""
    rng = np.random.default_rng(7 + digits)
    M, N, K = 130, 40, 200
    gaps = 2.0 ** -rng.integers(32, 51, (M, K))
    A = (1.0 - gaps) * rng.choice([-1.0, 1.0], (M, K)) * 2.0 ** rng.integers(-3, 4, (M, 1))
    A = A + 1j * (1.0 - gaps[::-1]) * rng.choice([-1.0, 1.0], (M, K))
    B = rng.standard_normal((K, N)) + 1j * (1.0 - 2.0 ** -rng.integers(32, 51, (K, N)))
    want = A @ B
    scale = np.abs(A) @ np.abs(B)
    got = ctx.hopf_tc_zgemm(A, B, 0, 0, digits=digits)
    rel = float(np.max(np.abs(got - want) / scale))
    assert rel <= 2.0 ** (-8 * digits + 5)


def test_rejects_bad_arguments(ctx):
    from paper_2403_04946_gb300 import binding
    A = np.ones((4, 4), dtype=complex)
    with pytest.raises(binding.HopfError) as e:
        ctx.hopf_tc_zgemm(A, A, digits=6)
    assert e.value.status == binding.HOPF_EINVAL
    with pytest.raises(binding.HopfError):
        ctx.hopf_tc_zgemm(A, A, digits=0)
