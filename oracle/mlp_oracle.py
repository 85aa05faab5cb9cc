"""Plain FP64 oracle of the learned planner's surrogate (test infrastructure only).

Sec. IV.C, Eq. nn_surrogate and Eq. nn_loss, with the workload's three-layer
form: z = (x - mu)/sigma, a1 = tanh(z W1 + b1), a2 = tanh(a1 W2 + b2),
f = a2 W3 + b3; loss = sum mask (f - y)^2 / sum mask.  Gradients by the chain
rule written out step by step; Adam with the usual bias correction.  The
parameter vector is flat in the order W1, b1, W2, b2, W3, b3 (row-major,
input index first), the layout of the library's parameters.
"""
import numpy as np


def unpack(p, F, H, O):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    out = []
    for shape in [(F, H), (H,), (H, H), (H,), (H, O), (O,)]:
        n = int(np.prod(shape))
        out.append(p[i:i + n].reshape(shape))
        i += n
    assert i == p.size
    return out


def forward(p, mu, sd, X, F, H, O):
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H, O)
    z = (np.asarray(X, np.float64) - mu) / sd
    a1 = np.tanh(z @ W1 + b1)
    a2 = np.tanh(a1 @ W2 + b2)
    return z, a1, a2, a2 @ W3 + b3


def loss_grad(p, mu, sd, X, Y, mask, F, H, O):
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H, O)
    z, a1, a2, f = forward(p, mu, sd, X, F, H, O)
    Y = np.asarray(Y, np.float64)
    M = np.ones_like(Y) if mask is None else np.asarray(mask, np.float64)
    n = M.sum()
    r = f - Y
    loss = float((M * r * r).sum() / n)
    g3 = 2.0 * M * r / n                    # d loss / d f
    dW3 = a2.T @ g3
    db3 = g3.sum(0)
    g2 = (g3 @ W3.T) * (1.0 - a2 * a2)      # through tanh of layer 2
    dW2 = a1.T @ g2
    db2 = g2.sum(0)
    g1 = (g2 @ W2.T) * (1.0 - a1 * a1)      # through tanh of layer 1
    dW1 = z.T @ g1
    db1 = g1.sum(0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad


def train_adam(p, mu, sd, X, Y, mask, F, H, O, epochs, lr, b1=0.9, b2=0.999, eps=1e-8):
    p = np.array(p, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    curve = []
    for t in range(1, epochs + 1):
        loss, g = loss_grad(p, mu, sd, X, Y, mask, F, H, O)
        curve.append(loss)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, np.array(curve)


def zscore(X):
    X = np.asarray(X, np.float64)
    mu = X.mean(0)
    sd = X.std(0)
    sd[sd <= 1e-6] = 1.0
    return mu, sd
