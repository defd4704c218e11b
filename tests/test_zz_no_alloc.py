"""dm_solve_band_noalloc, the allocation-free banded solve, against
dm_solve_band on two calls in a row.

Callers that cannot allocate device memory (real-time loops that cannot take
cudaMalloc's device-wide synchronisation, processes whose device memory is
held by another allocator) use the no-allocation entry point; it must give
the same answer as the allocating one, also when its fixed scratch array
still holds the previous call's data.  This file is collected last so that a
run stopping at the first failure has run everything else first."""
import numpy as np
import pytest

from test_gpu_band_solve import random_band_batch

pytestmark = pytest.mark.gpu


def _solve_both(sizes, seed):
    import torch
    from paper_2311_18126_gb300 import ensure_built, solve_band, solve_band_noalloc
    ensure_built()
    band, rhs, _ = random_band_batch(sizes, seed)
    d0 = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    tb = torch.tensor(band, device="cuda")
    tr = torch.tensor(rhs, device="cuda")
    ref = torch.empty_like(tr)
    out = torch.full_like(tr, float("nan"))
    solve_band(d0, sizes, tb, tr, ref)
    solve_band_noalloc(d0, sizes, tb, tr, out)
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_matches_allocating_solve_twice():
    # two different batches in a row: the second call sees the first call's
    # leftovers in the shared scratch array
    for sizes, seed in (([799, 197, 33, 32, 31, 11, 7], 1), ([40] * 64 + [150] * 9, 2)):
        ref, out = _solve_both(sizes, seed)
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_oversized_batch():
    import torch
    from paper_2311_18126_gb300 import DismechError, ensure_built, solve_band_noalloc
    from paper_2311_18126_gb300.dismech import NOALLOC_MAX_DOFS
    ensure_built()
    n = NOALLOC_MAX_DOFS + 1
    tb = torch.zeros((11, n), dtype=torch.float64, device="cuda")
    tr = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(DismechError) as ei:
        solve_band_noalloc([0], [n], tb, tr, torch.empty_like(tr))
    assert ei.value.code == 1 and "limit" in str(ei.value)


def test_noalloc_full_scratch_on_a_side_stream_then_a_smaller_batch():
    # exactly the fixed limit (2048 systems, 32768 DOFs, short and twisted
    # systems mixed), ordered on a non-default stream, then a much smaller
    # batch whose scratch regions still hold the first call's data
    import torch
    from paper_2311_18126_gb300 import ensure_built, solve_band, solve_band_noalloc
    from paper_2311_18126_gb300.dismech import NOALLOC_MAX_DOFS, NOALLOC_MAX_SYSTEMS
    ensure_built()
    big = [4] * 1536 + [40] * 256 + [64] * 256
    assert len(big) == NOALLOC_MAX_SYSTEMS and sum(big) == NOALLOC_MAX_DOFS
    side = torch.cuda.Stream()
    for sizes, seed in ((big, 3), ([799, 197, 33, 32, 31, 11, 7], 4)):
        band, rhs, _ = random_band_batch(sizes, seed)
        d0 = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        tb = torch.tensor(band, device="cuda")
        tr = torch.tensor(rhs, device="cuda")
        ref = torch.empty_like(tr)
        solve_band(d0, sizes, tb, tr, ref)
        out = torch.full_like(tr, float("nan"))
        side.wait_stream(torch.cuda.current_stream())
        solve_band_noalloc(d0, sizes, tb, tr, out, stream=side.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
