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
