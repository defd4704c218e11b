"""Warm-start network on the GPU (tcgen05 training and inference kernels)
against the FP64 CPU reference with the same bfloat16 rounding points."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _setup(M=256, n_in=40, n_out=4, seed=0):
    import torch
    from paper_2311_18126_gb300 import MLP, ensure_built
    ensure_built()
    net = MLP(n_in, n_out, seed=seed)
    rng = np.random.default_rng(seed)
    X = np.zeros((M, 64))
    X[:, :n_in] = rng.standard_normal((M, n_in))
    Xb = ref.bf16(X)
    Y = rng.standard_normal((M, n_out))
    tX = torch.tensor(Xb, dtype=torch.float32).to(torch.bfloat16).cuda()
    tY = torch.tensor(Y, dtype=torch.float32).cuda()
    return net, Xb, Y, tX, tY


def test_forward_matches_reference():
    import torch
    net, Xb, Y, tX, tY = _setup()
    out = torch.empty(tX.shape[0], 64, dtype=torch.float32, device="cuda")
    net.forward(tX, out)
    p = net.get_params().astype(np.float64)
    want = ref.forward(p, Xb, rounding=True)[-1]
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=2 ** -7, atol=2 ** -7 * np.abs(want).max())
    assert np.all(got[:, 4:] == 0.0)


def test_gradients_match_reference():
    import torch
    net, Xb, Y, tX, tY = _setup(M=384, seed=1)
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    loss = net.train_step(tX, tY, 0.0, grads=g)
    p = net.get_params().astype(np.float64)
    loss_ref, g_ref = ref.loss_and_grad(p, Xb, Y, 4, rounding=True)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    got = g.cpu().numpy().astype(np.float64)
    # element by element: both sides round operands to bfloat16 at the same
    # points but sum in a different order and precision (FP32 in tensor
    # memory), so an operand can land on the neighbouring bfloat16 value
    # (2^-7 relative); per entry the difference stays within 2^-5 of the
    # sum of the absolute values of its terms (first-order 2^-6 for the two
    # operands of a product, doubled for propagation through the layers
    # and the FP32 accumulation, K 2^-24 <= 2^-10 for K <= 16384)
    S = ref.grad_abs_scale(p, Xb, Y, 4)
    err = np.abs(got - g_ref)
    assert np.all(err <= 2.0 ** -5 * S + 1e-30), float(np.max(err / (S + 1e-300)))
    # and most entries agree to the FP32 accumulation alone
    assert np.mean(err <= 2.0 ** -10 * S + 1e-30) > 0.9
    o = 0
    for fi, fo in zip(ref.DIN, ref.DOUT):
        for n in (fo * fi, fo):
            a, b = got[o:o + n], g_ref[o:o + n]
            assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-12
            o += n


def test_training_reduces_loss():
    import torch
    net, Xb, Y, tX, tY = _setup(M=512, seed=2)
    # a learnable target: a smooth function of the inputs
    Xf = Xb[:, :40]
    T = np.stack([np.sin(Xf[:, 0]) + 0.5 * Xf[:, 1], Xf[:, 2] * Xf[:, 3], np.tanh(Xf[:, 4]),
                  0.3 * Xf[:, 5]], 1)
    tT = torch.tensor(T, dtype=torch.float32).cuda()
    l0 = net.train_step(tX, tT, 3e-3)
    for _ in range(300):
        last = net.train_step(tX, tT, 3e-3)
    assert last < 0.1 * l0


@pytest.mark.parametrize("M", [128, 256 * 152 + 384, 444544])
def test_fused_inference_equals_per_layer_gemms(M):
    """The fused 4-layer kernel (TMA, swizzled operands, activations in
    shared memory) against one GEMM launch per layer: the same BF16 rounding
    points, K blocks and tensor-core instruction shapes, so the outputs
    agree bit for bit; M spans one tile, several tiles per CTA with a
    ragged last round of tiles, and the bench's 444544 rows."""
    import torch
    net, Xb, Y, tX, tY = _setup(M=M, seed=3)
    a = torch.empty(M, 64, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    net.forward(tX, a)
    net.set_fused(False)
    net.forward(tX, b)
    net.set_fused(True)
    torch.cuda.synchronize()
    assert torch.equal(a, b), float((a - b).abs().max())


def test_async_inference_matches_synchronous():
    import torch
    net, Xb, Y, tX, tY = _setup(M=512, seed=4)
    a = torch.empty(512, 64, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    net.forward(tX, a)
    net.forward_async(tX, b)
    net.check()
    assert torch.equal(a, b)
