"""Host emulations (numpy, CPU) of arithmetic the solver kernels do with
integer tricks or blocked indexing, checked against plain definitions:

* the FP64 reciprocal: an FP32 seed built from the upper bits of d by
  integer operations (exponent rebiased by 1023 - 127), its FP32 reciprocal,
  moved back the same way, then one third-order step r (1 + e + e^2) with
  e = 1 - d r;
* the tiny-pivot test on the upper 32 bits of |D| and |J_jj| (exponent
  field minus 43, floored at 2^-126, ceiling 2^126) against
  |D| < 2^-43 |J_jj|;
* the blocked back substitution of a chain (blocks of 11 rows from the
  separator down, a sliding 22-slot buffer of running values, the z of row
  k - 11 brought in at row k, the unrolled step for blocks whose rows are
  all in [11, kstart)) against x_i = z_i - sum_d L[i+d][i] x_{i+d};
* the limb factor's small LU of the condensed block on the augmented
  matrix (the trailing update and the back substitution over (row, column)
  pairs, rows from a float reciprocal) against a dense LAPACK solve.
"""
import numpy as np

U32 = np.uint32


def _hi_lo(d):
    b = np.asarray(d, dtype=np.float64).view(np.uint64)
    return (b >> np.uint64(32)).astype(U32), (b & np.uint64(0xFFFFFFFF)).astype(U32)


def _seed(d):
    """FP32 seed of 1/d as the kernels form it (a correctly rounded FP32
    reciprocal stands in for the approximate instruction, whose error is
    within one unit in the last place)."""
    hi, lo = _hi_lo(d)
    fb = (hi & U32(0x80000000)) | (((hi & U32(0x7FFFFFFF)) - U32(0x38000000)) << U32(3)) | (lo >> U32(29))
    f = fb.view(np.float32)
    s = (np.float32(1.0) / f).astype(np.float32)
    sb = s.view(U32)
    h2 = (sb & U32(0x80000000)) | (((sb & U32(0x7FFFFFFF)) >> U32(3)) + U32(0x38000000))
    l2 = (sb << U32(29)).astype(U32)
    r = ((h2.astype(np.uint64) << np.uint64(32)) | l2.astype(np.uint64)).view(np.float64)
    return f, s, r


def test_reciprocal_seed_and_third_order_step():
    rng = np.random.default_rng(0)
    d = np.concatenate([10.0 ** rng.uniform(-37, 37, 100000), -(10.0 ** rng.uniform(-37, 37, 2000)),
                        np.array([2.0 ** -126, 2.0 ** 125.99, 1.0, 3.0, 0.1, -7.5])])
    f, s, r = _seed(d)
    # the FP32 number is d truncated to 23 mantissa bits
    assert np.all(np.abs(f.astype(np.float64) / d - 1.0) < 2.0 ** -23)
    # converting the FP32 reciprocal back is exact
    assert np.array_equal(r, s.astype(np.float64))
    assert np.max(np.abs(r * d - 1.0)) < 2.0 ** -22
    # one third-order step: the error is the seed's cubed, below FP64 rounding
    e = 1.0 - d * r
    rn = r + r * (e + e * e)
    assert np.max(np.abs(rn * d - 1.0)) <= 4 * np.finfo(np.float64).eps


def _hiword(x):
    return (np.asarray(x, dtype=np.float64).view(np.uint64) >> np.uint64(32)).astype(np.int64) & 0x7FFFFFFF


def _pivot_bad(D, J):
    thr = np.maximum(_hiword(J) - (43 << 20), (1023 - 126) << 20)
    h = _hiword(D)
    return (h < thr) | (h >= (1023 + 126) << 20)


def test_integer_pivot_test_matches_relative_threshold():
    rng = np.random.default_rng(1)
    J = 10.0 ** rng.uniform(-6, 6, 200000) * rng.choice([-1.0, 1.0], 200000)
    D = J * 10.0 ** rng.uniform(-16, -10, 200000) * rng.choice([-1.0, 1.0], 200000)
    ref = np.abs(D) < 2.0 ** -43 * np.abs(J)
    bad = _pivot_bad(D, J)
    # exact but for ties in the upper 32 bits (relative 2^-20)
    ratio = np.abs(D) / (2.0 ** -43 * np.abs(J))
    differ = bad != ref
    assert np.all(np.abs(ratio[differ] - 1.0) < 2.0 ** -19)
    assert differ.sum() <= 2
    # zero, subnormal, infinite and NaN pivots fail; ordinary ones pass
    for v in (0.0, -0.0, 1e-310, np.inf, -np.inf, np.nan, 2.0 ** 127):
        assert _pivot_bad(np.array([v]), np.array([1.0]))[0]
    assert not _pivot_bad(np.array([0.5]), np.array([1.0]))[0]
    assert not _pivot_bad(np.array([-3e4]), np.array([2e5]))[0]


def _back_reference(L, z, xs, kstart, nrows):
    x = np.zeros(nrows + 20)
    for i in range(10):
        if kstart + i < nrows:
            x[kstart + i] = xs[i]
    for i in range(kstart - 1, -1, -1):
        v = z[i]
        for d in range(1, 11):
            if i + d < min(nrows, kstart + 10):
                v -= L[i + d, d] * x[i + d]
        x[i] = v
    return x[:kstart]


def _back_blocked(L, z, xs, kstart, nrows, gfast=None):
    def stage(k0, full):
        buf = np.zeros(121)
        for e in range(121):
            u, d = divmod(e, 11)
            kk = k0 - u
            if full:  # every entry exists: no tests
                assert 11 <= kk < kstart
                buf[e] = z[kk - 11] if d == 0 else L[kk, d]
            elif kk >= 0:
                if d == 0:
                    if 0 <= kk - 11 < kstart:
                        buf[e] = z[kk - 11]
                elif kk < nrows and 0 <= kk - d < kstart:
                    buf[e] = L[kk, d]
        return buf

    Z = np.full(23, np.nan)
    for i in range(10):
        Z[i] = xs[9 - i]
    Z[10] = z[kstart - 1] if kstart >= 1 else 0.0
    nblk = (kstart + 20) // 11
    if gfast is None:
        gfast = min((kstart - 12) // 11 + 1 if kstart >= 12 else 1, nblk)
    x = np.zeros(nrows + 20)
    bufs = [stage(kstart + 9, False), None]
    for g in range(nblk):
        k0 = kstart + 9 - 11 * g
        cur = bufs[g & 1]
        if g + 1 < nblk:
            bufs[(g + 1) & 1] = stage(k0 - 11, g + 1 < gfast)
        for u in range(11):
            k = k0 - u
            xk = Z[u]
            if 1 <= g < gfast:  # unrolled step
                x[k] = xk
                for d in range(1, 11):
                    Z[u + d] = -cur[11 * u + d] * xk + Z[u + d]
                Z[u + 11] = cur[11 * u]
            else:
                act = 0 <= k < nrows
                if act and k < kstart:
                    x[k] = xk
                if act:
                    for d in range(1, 11):
                        if 0 <= k - d < kstart:
                            Z[u + d] = -cur[11 * u + d] * xk + Z[u + d]
                if 0 <= k - 11 < kstart:
                    Z[u + 11] = cur[11 * u]
        Z[0:11] = Z[11:22].copy()
    return x[:kstart]


def test_blocked_back_substitution_matches_direct():
    rng = np.random.default_rng(2)
    for n in (7, 11, 12, 21, 22, 23, 31, 32, 33, 40, 79, 197, 799):
        twist = n >= 32
        m = (n - 10) // 2 if twist else n
        for kstart in ([m, n - m - 10] if twist else [n]):
            rows = kstart + 10 if twist else n  # a chain sees its rows up to the separator
            L = rng.standard_normal((n + 20, 11)) * 0.3
            z = rng.standard_normal(n + 20)
            xs = rng.standard_normal(10) if twist else np.zeros(10)
            ref = _back_reference(L, z, xs, kstart, rows)
            for gfast in (None, 1):  # with and without the unrolled blocks
                got = _back_blocked(L, z, xs, kstart, rows, gfast)
                np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def _small_lu_solve(M, n, nrhs):
    """The condensed block's LU as the warp runs it on the augmented matrix
    [A | B] (n x (n + nrhs)): partial pivoting, reciprocal pivots, the
    trailing update over (row, column) pairs whose row comes from a float
    reciprocal, the back substitution column by column of U over (row,
    right-hand side) pairs."""
    M = M.copy()
    dinv = np.zeros(n)
    for j in range(n):
        bi = j + int(np.argmax(np.abs(M[j:, j])))
        M[[j, bi]] = M[[bi, j]]
        rp = 1.0 / M[j, j]
        dinv[j] = rp
        lm = M[:, j] * rp
        wdt = n + nrhs - j - 1
        iw = np.float32(1.0) / np.float32(wdt)
        for e in range((n - j - 1) * wdt):
            r = int((np.float32(e) + np.float32(0.5)) * iw)
            assert r == e // wdt  # the float row is exact here
            i, c = j + 1 + r, j + 1 + e - r * wdt
            M[i, c] = -lm[i] * M[j, c] + M[i, c]
    ir = np.float32(1.0) / np.float32(nrhs)
    for i in range(n - 1, -1, -1):
        M[i, n:] *= dinv[i]
        for e in range(i * nrhs):
            k = int((np.float32(e) + np.float32(0.5)) * ir)
            assert k == e // nrhs
            c = e - k * nrhs
            M[k, n + c] = -M[k, i] * M[i, n + c] + M[k, n + c]
    return M[:, n:]


def test_small_lu_pairs_match_dense_solve():
    rng = np.random.default_rng(3)
    for n in range(1, 11):
        for nrhs in (1, 2, 9, 17):
            A = rng.standard_normal((n, n)) + 0.1 * np.eye(n)
            B = rng.standard_normal((n, nrhs))
            got = _small_lu_solve(np.hstack([A, B]), n, nrhs)
            np.testing.assert_allclose(got, np.linalg.solve(A, B), rtol=1e-9, atol=1e-9)
