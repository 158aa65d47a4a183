"""FP64 NumPy oracle of the lateral-correction surrogate network.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs).  It restates
the network the CUDA kernels train and evaluate, in double precision, with
an analytic backward pass:

    x = taps - 1 (48 nearest-voxel densities),  z1 = x W1 + b1,  h1 = silu(z1),
    z2 = h1 W2 + b2,  h2 = silu(z2),  y = h2 W3 + b3,  densities = 1 + y,
    loss = sum over samples and outputs of (y - (t - 1))^2 / (3 n).

Parameters are packed as W1[48][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3].
"""
import numpy as np

SHAPES = [(48, 64), (64,), (64, 64), (64,), (64, 3), (3,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)   # 7491


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def forward(theta, X):
    """Effective densities [n, 3] from nearest-voxel taps [n, 48]."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(X, np.float64) - 1.0
    h1 = silu(x @ W1 + b1)
    h2 = silu(h1 @ W2 + b2)
    return 1.0 + h2 @ W3 + b3


def loss_grad(theta, X, T):
    """(loss, gradient [7491]) of the mean squared error, by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(X, np.float64) - 1.0
    t = np.asarray(T, np.float64) - 1.0
    n = x.shape[0]
    z1 = x @ W1 + b1
    s1 = 1.0 / (1.0 + np.exp(-z1))
    h1 = z1 * s1
    z2 = h1 @ W2 + b2
    s2 = 1.0 / (1.0 + np.exp(-z2))
    h2 = z2 * s2
    y = h2 @ W3 + b3
    r = y - t
    loss = float((r * r).sum() / (3.0 * n))
    dy = 2.0 * r / (3.0 * n)
    gW3 = h2.T @ dy
    gb3 = dy.sum(0)
    dz2 = (dy @ W3.T) * (s2 * (1.0 + z2 * (1.0 - s2)))
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (s1 * (1.0 + z1 * (1.0 - s1)))
    gW1 = x.T @ dz1
    gb1 = dz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g
