"""FP64 reference of the cost-model MLP -- TEST INFRASTRUCTURE ONLY.

Plain numpy: layers in -> H -> H -> H -> 1, ReLU on the hidden layers,
y = x W + b per layer; loss = mean squared error.  The flat parameter
vector is [W1, b1, W2, b2, W3, b3, W4, b4] with each W row-major
(inputs x outputs).  Backward pass written out by the chain rule.  Pinned by
central finite differences (tests/test_oracle_mlp.py)."""
import numpy as np


def shapes(n_in, hidden, layers=4):
    dims = [n_in] + [hidden] * (layers - 1) + [1]
    return [(dims[i], dims[i + 1]) for i in range(layers)]


def unpack(p, n_in, hidden):
    out, k = [], 0
    for i, o in shapes(n_in, hidden):
        W = p[k:k + i * o].reshape(i, o)
        k += i * o
        b = p[k:k + o]
        k += o
        out.append((W, b))
    assert k == p.size
    return out


def forward(p, x, hidden):
    p = np.asarray(p, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    layers = unpack(p, x.shape[1], hidden)
    acts = [x]
    h = x
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(h)
    return h[:, 0], acts


def loss_and_grad(p, x, t, hidden):
    """MSE loss and its gradient with respect to the flat parameters."""
    p = np.asarray(p, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    y, acts = forward(p, x, hidden)
    n = y.shape[0]
    loss = float(np.mean((y - t) ** 2))
    layers = unpack(p, x.shape[1], hidden)
    dz = (2.0 * (y - t) / n)[:, None]          # d loss / d output
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a_in = acts[li]
        grads.append((a_in.T @ dz, dz.sum(axis=0)))
        if li > 0:
            dz = (dz @ W.T) * (acts[li] > 0)   # ReLU of the previous layer
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.ravel())
        flat.append(db.ravel())
    return loss, np.concatenate(flat)
