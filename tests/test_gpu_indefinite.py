"""The pivot-free banded solves where the Jacobian J = M/dt^2 - dF/dq is not
positive definite (Sec. III-C, Eq. 16): a compressed, buckling rod and the
paper's large-step cantilevers (Table II, a1 and a2), per step against the
oracle (banded LU with partial pivoting); indefinite banded systems against
LAPACK; and a pivot that is tiny against its row, which the library must
report as DM_ERR_DEGENERATE instead of returning an inaccurate solution."""
import numpy as np
import pytest

from oracle import OracleSystems
from test_gpu_parity import _assert_close, _gpu

pytestmark = pytest.mark.gpu


def _indefinite_band_batch(sizes, seed):
    """Symmetric banded systems (half bandwidth 10) with diagonal entries of
    both signs, diagonally dominant so that elimination in order is stable."""
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
        A += np.diag(rng.choice([-1.0, 1.0], n) * (25.0 + 5.0 * rng.random(n)))
        for i in range(n):
            for d in range(0, min(i, 10) + 1):
                band[d, off + i] = A[i, i - d]
        dense.append(A)
        off += n
    return band, rng.standard_normal(ntot), dense


def _solvers():
    from paper_2311_18126_gb300 import solve_band, solve_band_noalloc
    from paper_2311_18126_gb300.dismech import solve_band_partitioned
    return [("band", solve_band), ("noalloc", solve_band_noalloc),
            ("partitioned", lambda d0, nd, b, r, x: solve_band_partitioned(d0, nd, b, r, x, 64))]


@pytest.mark.parametrize("sizes", [[7, 31, 33, 197, 799], [300, 41, 1500]])
def test_indefinite_band_systems_match_lapack(sizes):
    import torch
    from paper_2311_18126_gb300 import ensure_built
    ensure_built()
    band, rhs, dense = _indefinite_band_batch(sizes, 7 + len(sizes))
    for A in dense:
        ev = np.linalg.eigvalsh(A)
        assert ev[0] < 0 < ev[-1]
    d0 = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    tb = torch.tensor(band, device="cuda")
    tr = torch.tensor(rhs, device="cuda")
    for name, solve in _solvers():
        tx = torch.full_like(tr, float("nan"))
        solve(d0, sizes, tb, tr, tx)
        x = tx.cpu().numpy()
        off = 0
        for n, A in zip(sizes, dense):
            ref = np.linalg.solve(A, rhs[off:off + n])
            np.testing.assert_allclose(x[off:off + n], ref, rtol=1e-11, atol=1e-13,
                                       err_msg=name)
            off += n


def test_tiny_pivot_is_reported_as_degenerate():
    import torch
    from paper_2311_18126_gb300 import DismechError, ensure_built
    ensure_built()
    # a 100-row system whose leading 2 x 2 block is singular up to 1e-15 of
    # its diagonal: the second pivot is 1e-15 |J_11|, below 1e-13 |J_11|
    n = 100
    A = np.eye(n) * 4.0
    A[0, 0] = A[1, 1] = 1.0
    A[1, 0] = A[0, 1] = 1.0
    A[1, 1] += 1e-15
    band = np.zeros((11, n))
    for i in range(n):
        for d in range(0, min(i, 10) + 1):
            band[d, i] = A[i, i - d]
    tb = torch.tensor(band, device="cuda")
    tr = torch.ones(n, dtype=torch.float64, device="cuda")
    for name, solve in _solvers():
        with pytest.raises(DismechError) as ei:
            solve([0], [n], tb, tr, torch.empty_like(tr))
        assert ei.value.code == 4, name
    # the same system with a well-separated second pivot is solved
    A[1, 1] = 2.0
    band[0, 1] = 2.0
    tb = torch.tensor(band, device="cuda")
    for name, solve in _solvers():
        tx = torch.empty_like(tr)
        solve([0], [n], tb, tr, tx)
        np.testing.assert_allclose(tx.cpu().numpy(), np.linalg.solve(A, np.ones(n)),
                                   rtol=1e-13, err_msg=name)


def _column(N=21, L=0.3, h=1e-3, E=1e6, dt=0.1):
    # a rod standing on its clamped lower end, about five times longer than
    # its self-buckling length 1.986 (EI / (rho A g))^(1/3) = 5.9 cm, with a
    # small lateral imperfection; at dt = 0.1 s the inertia M/dt^2 no longer
    # stabilises it and it collapses under its own weight
    z = np.linspace(0.0, L, N)
    x = np.stack([1e-4 * np.sin(np.pi * z / (2 * L)), np.zeros(N), z], 1)
    fixed = np.zeros(4 * N - 1, np.uint8)
    fixed[:8] = 1
    desc = dict(nodes_per_rod=[N], x0=x, E=[E], nu=[0.5], rho=[1000.0], radius=[h],
                fixed=fixed)
    return desc, dict(dt=dt, tol=1e-10, max_iter=100, g=(0.0, 0.0, -9.81), eta=0.0)


def test_buckling_column_per_step_with_indefinite_jacobian():
    desc, params = _column()
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    s = ora.systems[0]
    npr = desc["nodes_per_rod"]
    neg, its = [], []
    for k in range(8):
        # negative eigenvalues of J at the start of the step (symmetric: no
        # friction, no contact)
        _, _, J = ora.residual(s, s.q, s.q, s.v, need_jac=True)
        neg.append(int((np.linalg.eigvalsh(J.numpy()) < 0).sum()))
        gpu.step(1)
        st = ora.step(1)
        assert st[0][0] == 0, st
        its.append(st[0][1])
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 0.3, 1e-10)
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
    assert max(neg) >= 5, neg          # strongly indefinite along the way
    assert max(its) >= 10, its         # and Newton works for it


def _table2_cantilever(E, dt):
    # Table II: N = 201, h = 2 cm, rho = 500, L = 1 m, no gravity; free
    # vibration from an initial tip velocity of 5 mm/s (quadratic profile)
    N, L = 201, 1.0
    x = np.zeros((N, 3))
    x[:, 0] = np.linspace(0.0, L, N)
    v = np.zeros((N, 3))
    v[:, 2] = 5e-3 * (x[:, 0] / L) ** 2
    fixed = np.zeros(4 * N - 1, np.uint8)
    fixed[:8] = 1
    desc = dict(nodes_per_rod=[N], x0=x, v0=v, E=[E], nu=[0.5], rho=[500.0], radius=[0.02],
                fixed=fixed)
    return desc, dict(dt=dt, tol=1e-10, max_iter=100, g=(0.0, 0.0, 0.0), eta=0.0)


@pytest.mark.parametrize("E,dt", [(1e5, 0.5), (1e7, 0.05)])
@pytest.mark.parametrize("integ", ["be", "midpoint"])
def test_table2_cantilever_large_steps_per_step(E, dt, integ):
    desc, params = _table2_cantilever(E, dt)
    params = dict(params, integrator=integ)
    gpu = _gpu(desc, params)
    ora = OracleSystems(desc, params)
    npr = desc["nodes_per_rod"]
    for k in range(4):
        gpu.step(1)
        st = ora.step(1)
        assert st[0][0] == 0, st
        qg, vg = gpu.get_state()
        qo, vo = ora.get_state()
        _assert_close(qg, qo, npr, 1.0, 1e-10)
        d1, beta = ora.get_frames()
        gpu.set_state(qo, vo)
        gpu.set_frames(d1, beta)
