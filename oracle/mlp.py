"""FP64 reference for the warm-start MLP (8 -> 128 -> 128 -> 1, ReLU), TEST INFRASTRUCTURE ONLY.

Same parameter layout as the library: W1[128][8], b1[128], W2[128][128], b2[128], W3[128], b3.
The forward pass takes the parameters as given (pass the BF16-rounded values to mirror the device's
forward); inputs are normalised as (x - mean) / scale.  The loss is (1/N) sum_i (y_i - target_i)^2.
"""
import numpy as np

IN, H = 8, 128
SIZES = [("W1", H * IN), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H), ("b3", 1)]
COUNT = sum(s for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, size in SIZES:
        out[name] = p[o:o + size]
        o += size
    out["W1"] = out["W1"].reshape(H, IN)
    out["W2"] = out["W2"].reshape(H, H)
    return out


def forward(p, X, norm):
    q = unpack(p)
    Xn = (np.asarray(X, np.float64) - norm[:IN]) / norm[IN:]
    z1 = Xn @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ q["W3"] + q["b3"][0]
    return y, (Xn, z1, h1, z2, h2)


def loss_and_gradient(p, X, target, norm):
    """Mean squared error and its gradient with respect to the flat parameter vector (chain rule)."""
    q = unpack(p)
    y, (Xn, z1, h1, z2, h2) = forward(p, X, norm)
    N = len(y)
    r = y - np.asarray(target, np.float64)
    dy = 2.0 * r / N
    gW3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    dz2 = np.outer(dy, q["W3"]) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ q["W2"]) * (z1 > 0)
    gW1 = dz1.T @ Xn
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return float(np.mean(r ** 2)), g
