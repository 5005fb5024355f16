"""The arithmetic claims behind the sliced contraction, checked on an integer
model of it (numpy; no GPU, no library code): the error-free slicing of
Ozaki, Ogita, Oishi and Rump (2012) with balanced base-256 digits.

- Digits: x / 2^e (|x| < 2^e) rounded to 8 S fractional bits, then balanced
  base-256 digits; the first lies in [-256, 256], the others in [-128, 127],
  so each is exact in bf16 (8 significant bits), and the digits reconstruct
  x within 2^(e - 8 S - 1).
- Exact accumulation: over a real contraction length of 256 the level-2 sum
  (first digits) and the level-3 sum (first x second digits) stay within
  2^24 in magnitude even at the digits' bounds, so FP32 accumulation of
  integers is exact.
- Accuracy: with five slices per operand and levels up to 6, a complex
  product formed from the slices agrees with FP64 to about 2^-40 of the
  row and column scales; with four slices (the adjoint's products), 2^-33.
"""
import numpy as np


def digits(x, e, S):
    """Balanced base-256 digits of x / 2^e, S of them (first most significant)."""
    N = np.rint(np.ldexp(x, 8 * S - e)).astype(np.int64)
    out = []
    for _ in range(S - 1):
        d = ((N + 128) & 255) - 128
        out.append(d)
        N = (N - d) >> 8
    out.append(N)
    return out[::-1]  # d_1 .. d_S


def row_exponent(a):
    m = np.abs(a).max(axis=-1, keepdims=True)
    _, e = np.frexp(m)
    return np.where(m > 0, e, 0)


def test_digit_ranges_and_reconstruction():
    rng = np.random.default_rng(1)
    for S in (4, 5):
        x = rng.standard_normal((64, 300)) * np.exp(rng.uniform(-20, 20, (64, 1)))
        x[:, 0] = np.sign(x[:, 0]) * np.abs(x).max(axis=1)  # the largest magnitude in every row
        e = row_exponent(x)
        d = digits(x, e, S)
        assert np.all(np.abs(d[0]) <= 256)
        for di in d[1:]:
            assert np.all((di >= -128) & (di <= 127))
        recon = sum(di.astype(np.float64) * 2.0 ** (-8 * (i + 1)) for i, di in enumerate(d))
        err = np.abs(np.ldexp(recon, e) - x)
        assert np.all(err <= np.ldexp(1.0, e - 8 * S - 1) * (1 + 1e-12))


def test_level_sums_fit_fp32_exactly_at_length_256():
    # digits at their bounds: first 256, second 128 (or -128), over 256 real terms
    K = 256
    d1 = np.full(K, 256, dtype=np.int64)
    d2 = np.full(K, 128, dtype=np.int64)
    level2 = int(np.dot(d1, d1))
    level3 = int(np.dot(d1, d2) + np.dot(d2, d1))  # in units of 2^-8
    assert abs(level2) <= 2 ** 24 and abs(level3) <= 2 ** 24
    # every partial sum is an integer no larger than the total: exact in FP32
    for v in (np.cumsum(d1 * d1), np.cumsum(d1 * d2 * 2)):
        assert np.all(np.float32(v).astype(np.int64) == v)


def _sliced_complex_product(W, D, S, levels):
    """V = W D through the slices, complex as one real product of twice the
    length: [Wr | Wi] times [[Dr, Di], [-Di, Dr]]; pairs i + j <= levels."""
    M, K = W.shape
    A = np.concatenate([W.real, W.imag], axis=1)                      # M x 2K
    Br = np.concatenate([D.real, -D.imag], axis=0)                    # 2K x N (Re V)
    Bi = np.concatenate([D.imag, D.real], axis=0)                     # 2K x N (Im V)
    ea = row_exponent(A)                                              # per row of W
    eb = row_exponent(np.concatenate([Br, Bi], axis=0).T).T           # per string of D
    da = digits(A, ea, S)
    dr, di = digits(Br.T, eb.T, S), digits(Bi.T, eb.T, S)
    vr = np.zeros((M, D.shape[1]))
    vi = np.zeros((M, D.shape[1]))
    for i in range(S):
        for j in range(S):
            if i + j + 2 > levels:
                continue
            w = 2.0 ** (-8 * (i + j + 2))
            vr += w * (da[i] @ dr[j].T)   # integer products, exact in int64 and float64 here
            vi += w * (da[i] @ di[j].T)
    scale = np.ldexp(1.0, ea + eb)
    return (vr + 1j * vi) * scale, scale


def test_sliced_product_accuracy():
    rng = np.random.default_rng(2)
    M, K, N = 40, 120, 50
    W = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * np.exp(rng.uniform(-3, 3, (M, 1)))
    D = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * np.exp(rng.uniform(-3, 3, (1, N)))
    exact = W @ D
    for S, bound in ((5, 2.0 ** -40), (4, 2.0 ** -33)):  # observed 2^-44.3, 2^-36.5; three slices give 2^-28.7
        V, scale = _sliced_complex_product(W, D, S, S + 1)
        rel = np.abs(V - exact) / (scale * 2 * K)   # relative to the row x string scale times the length
        assert rel.max() < bound, (S, rel.max())
