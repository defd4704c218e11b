"""Plain FP64 reference of the warm-start network (no counterpart in the
paper; the network only predicts the Newton initial guess).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A 4-layer perceptron, widths 64 -> 256 -> 256 -> 256 -> 64 (input and output
padded to 64), ReLU on the hidden layers, mean squared error on the first
``n_out`` outputs.  With ``bf16=True`` the forward and backward passes round
to bfloat16 at the same points as the tensor-core kernels (operands of every
product, hidden activations, output and hidden-layer gradients); products
themselves are exact in FP64.
"""
import numpy as np

DIN = (64, 256, 256, 256)
DOUT = (256, 256, 256, 64)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    """Flat parameter vector -> list of (W [out][in], b [out])."""
    out, o = [], 0
    for fi, fo in zip(DIN, DOUT):
        W = params[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = params[o:o + fo]
        o += fo
        out.append((np.asarray(W, np.float64), np.asarray(b, np.float64)))
    return out


def forward(params, X, rounding=False):
    r = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    layers = unpack(params)
    acts = [r(X)]
    for l, (W, b) in enumerate(layers):
        z = acts[-1] @ r(W).T + b
        if l < len(layers) - 1:
            acts.append(r(np.maximum(z, 0.0)))
        else:
            acts.append(np.asarray(z, np.float32).astype(np.float64) if rounding else z)
    return acts


def loss_and_grad(params, X, Y, n_out, rounding=False):
    """MSE on the first n_out outputs and its gradient (flat layout)."""
    r = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    layers = unpack(params)
    acts = forward(params, X, rounding)
    M = X.shape[0]
    out = acts[-1]
    d = np.zeros_like(out)
    diff = out[:, :n_out] - Y[:, :n_out]
    loss = float(np.mean(diff ** 2))
    d[:, :n_out] = 2.0 * diff / (M * n_out)
    if rounding:
        d = np.asarray(d, np.float32).astype(np.float64)
    grads = [None] * len(layers)
    g = d
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gb = g.sum(0)
        gW = r(g).T @ acts[l]
        grads[l] = (gW, gb)
        if l > 0:
            dA = r(r(g) @ r(W))
            g = np.where(acts[l] > 0, dA, 0.0)
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat


def grad_abs_scale(params, X, Y, n_out):
    """Per gradient entry, the sum of the absolute values of the terms that
    make it up: the backward pass of ``loss_and_grad`` (with the bfloat16
    rounding points) run on |W|, |activations| and |output gradient|, ReLU
    masks of the rounded forward pass.  An element-wise error scale for a
    kernel that rounds at the same points but sums in another order and
    precision: moving one operand of a product to a neighbouring bfloat16
    value changes the product by at most 2^-7 of its magnitude."""
    layers = unpack(params)
    acts = forward(params, X, rounding=True)
    M = X.shape[0]
    out = acts[-1]
    d = np.zeros_like(out)
    d[:, :n_out] = np.abs(2.0 * (out[:, :n_out] - Y[:, :n_out]) / (M * n_out))
    grads = [None] * len(layers)
    g = d
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = g.T @ np.abs(acts[l])
        grads[l] = (gW, g.sum(0))
        if l > 0:
            g = np.where(acts[l] > 0, g @ np.abs(bf16(W)), 0.0)
    return np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
