"""The contraction kernels of the mixed-precision form against FP64 products formed on the host:
the tensor-core one (tcgen05, BF16 digit planes, FP32 accumulators in tensor memory; slices 2..4)
and the split-FP32 CUDA-core one of the small contractions (slices 1).

The split writes each row of op(A) and column of op(B), scaled by its own power of two, as S
balanced base-256 digits; integer-valued inputs that fit in 8S-1 bits are therefore represented
exactly and their products summed exactly, which makes the first test bit-exact: any mistake in
the operand layout, the matrix descriptors, the transposes or the ragged tile edges shows there.
The others check the stated bound, error <= 2^-(8S-1) k max_l |a_il| max_l |b_lj| per element,
with a factor 2 of margin."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_10270_gb300 import build as B
    B.build()
    from paper_1803_10270_gb300 import htgpu
    htgpu.load()
    return htgpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x.reshape(-1, order="F"))).cuda()


def _run(G, A, B, tA, tB, slices, alpha=1.0, beta=0.0, C0=None, colscale=None):
    """op(A) op(B) through the entry point; A and B are the STORED arrays (transposed when tA/tB)."""
    import torch
    m = A.shape[1] if tA else A.shape[0]
    k = A.shape[0] if tA else A.shape[1]
    n = B.shape[0] if tB else B.shape[1]
    Cd = _dev(C0 if C0 is not None else np.full((m, n), np.nan))
    cs = torch.from_numpy(colscale).cuda() if colscale is not None else None
    rc = G.selftest_gemm_mixed(_dev(A), _dev(B), Cd, m, n, k, A.shape[0], B.shape[0], m, tA, tB, alpha, beta,
                               cs, slices=slices)
    assert rc == G.HT_OK
    torch.cuda.synchronize()
    return Cd.cpu().numpy().reshape(m, n, order="F")


def _op(X, t):
    return X.T if t else X


@pytest.mark.parametrize("slices", [1, 2, 3, 4])
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_integer_inputs_are_exact(G, slices, tA, tB):
    """m = 200, n = 150 (two ragged tiles each way), k = 70 (three ragged stages of 32):
    integers in [-100, 100] fit every split (and their sums, below 2^24, the FP32 high part of the
    split-FP32 form), so C must equal the integer product exactly."""
    rng = np.random.default_rng(10 * slices + 2 * tA + tB)
    m, n, k = 200, 150, 70
    A = rng.integers(-100, 101, (m, k)).astype(np.float64)
    B = rng.integers(-100, 101, (k, n)).astype(np.float64)
    A[7, :] = 0.0                      # a zero row
    B[:, 3] = 0.0                      # a zero column
    A[11, :] = np.where(A[11, :] != 0, 1.0, 0.0)
    got = _run(G, _op(A, tA).copy(), _op(B, tB).copy(), tA, tB, slices)
    np.testing.assert_array_equal(got, A @ B)


@pytest.mark.parametrize("slices", [2, 3, 4])
def test_random_inputs_within_split_bound(G, slices):
    """Values spanning 10 decades within rows and columns; k = 500 (16 stages, group sums beyond
    2^24 for the higher digit groups)."""
    rng = np.random.default_rng(3 + slices)
    m, n, k = 260, 140, 500
    A = rng.standard_normal((m, k)) * np.exp(rng.uniform(-11.5, 11.5, (m, k)))
    B = rng.standard_normal((k, n)) * np.exp(rng.uniform(-3, 3, (k, n)))
    got = _run(G, A, B, 0, 0, slices)
    ref = A @ B
    bound = 2.0 ** -(8 * slices - 1) * k * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]
    ratio = (np.abs(got - ref) / bound).max()
    print(f"slices {slices}: max error / bound = {ratio:.3f}")
    assert ratio <= 2.0


def test_alpha_beta_colscale_and_batch(G):
    """C[b] = alpha op(A[b]) op(B[b]) diag(s) + beta C[b] over a batch with strides (the
    projection form Y = E Z S^-1 of the truncation), four slices."""
    import torch
    rng = np.random.default_rng(21)
    m, n, k, nb = 90, 40, 33, 5
    lda, ldb, ldc = m + 3, k + 1, m + 2
    sA, sB, sC = lda * k + 7, ldb * n + 5, ldc * n + 1
    Ab = rng.standard_normal(sA * nb)
    Bb = rng.standard_normal(sB * nb)
    Cb = rng.standard_normal(sC * nb)
    s = rng.uniform(0.5, 2.0, n) * 1e3
    alpha, beta = -0.75, 0.5
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (Ab, Bb, Cb))
    rc = G.selftest_gemm_mixed(Ad, Bd, Cd, m, n, k, lda, ldb, ldc, 0, 0, alpha, beta, torch.from_numpy(s).cuda(),
                               batch=nb, sA=sA, sB=sB, sC=sC, slices=4)
    assert rc == G.HT_OK
    got = Cd.cpu().numpy()
    for b in range(nb):
        A = Ab[b * sA: b * sA + lda * k].reshape(lda, k, order="F")[:m]
        B = Bb[b * sB: b * sB + ldb * n].reshape(ldb, n, order="F")[:k]
        C0 = Cb[b * sC: b * sC + ldc * n].reshape(ldc, n, order="F")
        ref = alpha * (A @ B) * s[None, :] + beta * C0[:m]
        G_ = got[b * sC: b * sC + ldc * n].reshape(ldc, n, order="F")
        bound = 2.0 ** -31 * k * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :] * abs(alpha) * s[None, :]
        assert (np.abs(G_[:m] - ref) / (bound + 1e-300)).max() <= 2.0 + 1e-6
        # rows between m and ldc are not touched
        np.testing.assert_array_equal(G_[m:], C0[m:])
    # the last batch entry's trailing elements beyond its stride are untouched
    np.testing.assert_array_equal(got[nb * sC:], Cb[nb * sC:])


def test_empty_inner_dimension_and_empty_output(G):
    """k = 0 gives C = beta C; m = 0 touches nothing."""
    import torch
    C0 = np.arange(12.0).reshape(3, 4)
    A = np.zeros((3, 1))
    B = np.zeros((1, 4))
    Cd = _dev(C0)
    rc = G.selftest_gemm_mixed(_dev(A), _dev(B), Cd, 3, 4, 0, 3, 1, 3, 0, 0, 1.0, 2.0, None, slices=4)
    assert rc == G.HT_OK
    np.testing.assert_array_equal(Cd.cpu().numpy().reshape(3, 4, order="F"), 2.0 * C0)
    rc = G.selftest_gemm_mixed(_dev(A), _dev(B), Cd, 0, 4, 1, 3, 1, 3, 0, 0, 1.0, 0.0, None, slices=4)
    assert rc == G.HT_OK
    np.testing.assert_array_equal(Cd.cpu().numpy().reshape(3, 4, order="F"), 2.0 * C0)


def test_split_fp32_within_bound(G):
    """The split-FP32 kernel (slices 1): values spanning 10 decades, k = 500 (32 ragged stages of
    16).  Per element the error must stay within the compensated dot product's worst-case bound
    (k^2 + 5k + 10) 2^-47 sum_l |a_il b_lj|, and within 2 (k/2 + 10) 2^-47 sum_l |a_il b_lj| (the
    size rounding errors of random sign give; a plain FP32 accumulation misses it by about 2^20)."""
    rng = np.random.default_rng(41)
    m, n, k = 70, 45, 500
    A = rng.standard_normal((m, k)) * np.exp(rng.uniform(-11.5, 11.5, (m, k)))
    B = rng.standard_normal((k, n)) * np.exp(rng.uniform(-3, 3, (k, n)))
    absAB = np.abs(A) @ np.abs(B)
    for tA, tB in ((0, 0), (0, 1), (1, 0), (1, 1)):
        got = _run(G, _op(A, tA).copy(), _op(B, tB).copy(), tA, tB, 1)
        err = np.abs(got - A @ B)
        worst = (k * k + 5 * k + 10) * 2.0 ** -47 * absAB
        typical = (k / 2 + 10) * 2.0 ** -47 * absAB
        print(f"split FP32, tA={tA} tB={tB}: max error / typical bound = {(err / typical).max():.3f}")
        assert (err <= worst).all()
        assert (err / typical).max() <= 2.0


def test_split_fp32_alpha_beta_colscale_and_batch(G):
    """The split-FP32 kernel on the projection form C[b] = alpha A[b] B[b] diag(s) + beta C[b]
    over a strided batch; rows past m and entries past the last stride untouched."""
    import torch
    rng = np.random.default_rng(22)
    m, n, k, nb = 37, 21, 19, 4
    lda, ldb, ldc = m + 3, k + 1, m + 2
    sA, sB, sC = lda * k + 7, ldb * n + 5, ldc * n + 1
    Ab = rng.standard_normal(sA * nb)
    Bb = rng.standard_normal(sB * nb)
    Cb = rng.standard_normal(sC * nb)
    s = rng.uniform(0.5, 2.0, n) * 1e3
    alpha, beta = -0.75, 0.5
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (Ab, Bb, Cb))
    rc = G.selftest_gemm_mixed(Ad, Bd, Cd, m, n, k, lda, ldb, ldc, 0, 0, alpha, beta, torch.from_numpy(s).cuda(),
                               batch=nb, sA=sA, sB=sB, sC=sC, slices=1)
    assert rc == G.HT_OK
    got = Cd.cpu().numpy()
    for b in range(nb):
        A = Ab[b * sA: b * sA + lda * k].reshape(lda, k, order="F")[:m]
        B = Bb[b * sB: b * sB + ldb * n].reshape(ldb, n, order="F")[:k]
        C0 = Cb[b * sC: b * sC + ldc * n].reshape(ldc, n, order="F")
        ref = alpha * (A @ B) * s[None, :] + beta * C0[:m]
        G_ = got[b * sC: b * sC + ldc * n].reshape(ldc, n, order="F")
        bound = (k / 2 + 10) * 2.0 ** -47 * (np.abs(A) @ np.abs(B)) * abs(alpha) * s[None, :] + 4e-16 * np.abs(ref)
        assert (np.abs(G_[:m] - ref) / bound).max() <= 2.0
        np.testing.assert_array_equal(G_[m:], C0[m:])
    np.testing.assert_array_equal(got[nb * sC:], Cb[nb * sC:])


def test_split_fp32_exponent_ranges(G):
    """The split's documented ranges: operands from 2^-74 up keep 48 significant bits (the
    (k^2 + 5k + 10) 2^-47 bound), operands between 2^-120 and 2^-75 keep only their FP32 high part
    (2^-23 relative per product), zeros stay exact; one matrix mixes all three."""
    rng = np.random.default_rng(77)
    m, n, k = 33, 29, 40
    mag = rng.choice([0.0, 1.0, 1.0], size=(m, k))
    expo = rng.uniform(-74.0, 100.0, (m, k))
    tiny = rng.random((m, k)) < 0.2
    expo[tiny] = rng.uniform(-120.0, -76.0, tiny.sum())
    A = mag * rng.choice([-1.0, 1.0], (m, k)) * np.exp2(expo) * rng.uniform(1.0, 2.0, (m, k))
    B = rng.standard_normal((k, n))
    got = _run(G, A, B, 0, 0, 1)
    ref = A @ B
    big = np.where(tiny, 0.0, np.abs(A))
    small = np.where(tiny, np.abs(A), 0.0)
    bound = ((k * k + 5 * k + 10) * 2.0 ** -47 * (big @ np.abs(B)) + 2.0 ** -23 * (small @ np.abs(B))
             + 2.0 ** -52 * np.abs(ref))
    assert (np.abs(got - ref) <= bound).all()
    zero_rows = (mag == 0.0).all(axis=1)
    if zero_rows.any():
        assert (got[zero_rows] == 0.0).all()
