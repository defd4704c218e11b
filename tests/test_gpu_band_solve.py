"""The public batched banded solve (dm_solve_band, the twisted LDL^T kernel
of the Newton step) against a dense LAPACK solve of the same systems."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def random_band_batch(sizes, seed):
    """Symmetric, diagonally dominant banded systems (half bandwidth 10),
    lower band in the [11, ntot] layout of the C ABI."""
    rng = np.random.default_rng(seed)
    ntot = int(sum(sizes))
    band = np.zeros((11, ntot))
    dense = []
    off = 0
    for n in sizes:
        A = np.zeros((n, n))
        for i in range(n):
            for j in range(max(0, i - 10), i):
                A[i, j] = A[j, i] = rng.standard_normal()
        A += np.diag(25.0 + 5.0 * rng.random(n))
        for i in range(n):
            for d in range(0, min(i, 10) + 1):
                band[d, off + i] = A[i, i - d]
        dense.append(A)
        off += n
    rhs = rng.standard_normal(ntot)
    return band, rhs, dense


@pytest.mark.parametrize("sizes", [[7, 11, 31, 32, 33, 197, 799], [40] * 64])
def test_band_solve_matches_dense(sizes):
    import torch
    from paper_2311_18126_gb300 import ensure_built, solve_band
    ensure_built()
    band, rhs, dense = random_band_batch(sizes, len(sizes))
    d0 = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    tb = torch.tensor(band, device="cuda")
    tr = torch.tensor(rhs, device="cuda")
    tx = torch.empty_like(tr)
    solve_band(d0, sizes, tb, tr, tx)
    x = tx.cpu().numpy()
    off = 0
    for n, A in zip(sizes, dense):
        ref = np.linalg.solve(A, rhs[off:off + n])
        np.testing.assert_allclose(x[off:off + n], ref, rtol=1e-12, atol=1e-14)
        off += n
    # the input band is not modified
    np.testing.assert_array_equal(tb.cpu().numpy(), band)


@pytest.mark.parametrize("part_rows", [21, 64, 512])
def test_partitioned_band_solve_matches_dense(part_rows):
    """The partitioned solve (interiors factored in parallel, Schur system on
    the separators) against a dense LAPACK solve, for systems shorter than
    one partition, exactly a few partitions and with ragged tails."""
    import torch
    from paper_2311_18126_gb300 import ensure_built
    from paper_2311_18126_gb300.dismech import solve_band_partitioned
    ensure_built()
    sizes = [7, 11, 31, 32, 33, 197, 799, 1500]
    band, rhs, dense = random_band_batch(sizes, 5)
    d0 = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    tb = torch.tensor(band, device="cuda")
    tr = torch.tensor(rhs, device="cuda")
    tx = torch.empty_like(tr)
    solve_band_partitioned(d0, sizes, tb, tr, tx, part_rows=part_rows)
    x = tx.cpu().numpy()
    off = 0
    for n, A in zip(sizes, dense):
        ref = np.linalg.solve(A, rhs[off:off + n])
        np.testing.assert_allclose(x[off:off + n], ref, rtol=1e-11, atol=1e-13)
        off += n


def _long_band(n, seed):
    rng = np.random.default_rng(seed)
    band = np.zeros((11, n))
    for d in range(1, 11):
        band[d, d:] = rng.standard_normal(n - d)
    band[0] = 25.0 + 5.0 * rng.random(n)
    return band, rng.standard_normal(n)


def test_partitioned_band_solve_long_systems():
    """Long systems (a 5000-node rod has 19999 DOFs): the partitioned solve
    against LAPACK's banded Cholesky and against the sequential twisted
    LDL^T; the device time of both is printed."""
    import scipy.linalg
    import torch
    from paper_2311_18126_gb300 import ensure_built, solve_band
    from paper_2311_18126_gb300.dismech import solve_band_partitioned
    ensure_built()
    sizes = [19999, 7999]
    parts = [_long_band(n, 10 + k) for k, n in enumerate(sizes)]
    band = np.concatenate([b for b, _ in parts], axis=1)
    rhs = np.concatenate([r for _, r in parts])
    d0 = [0, sizes[0]]
    tb = torch.tensor(band, device="cuda")
    tr = torch.tensor(rhs, device="cuda")
    tx = torch.empty_like(tr)
    ts = torch.empty_like(tr)
    times = {}
    for name, fn in (("partitioned", lambda: solve_band_partitioned(d0, sizes, tb, tr, tx)),
                     ("sequential", lambda: solve_band(d0, sizes, tb, tr, ts))):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 3
    print("long systems %s: partitioned %.3f ms, sequential %.3f ms per call (incl. scratch "
          "allocation)" % (sizes, times["partitioned"], times["sequential"]))
    x, xs = tx.cpu().numpy(), ts.cpu().numpy()
    off = 0
    for (b, r), n in zip(parts, sizes):
        ab = np.zeros((11, n))  # LAPACK lower form: ab[d, j] = A[j + d, j]
        for d in range(11):
            ab[d, :n - d] = b[d, d:]
        ref = scipy.linalg.solveh_banded(ab, r, lower=True)
        np.testing.assert_allclose(x[off:off + n], ref, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(x[off:off + n], xs[off:off + n], rtol=1e-10, atol=1e-12)
        off += n
