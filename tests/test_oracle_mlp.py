"""Pins of the oracle's smoothing-length MLP: forward against an independent
numpy restatement, gradient against central finite differences (FP64)."""
import numpy as np


def _params(rng, orc):
    P = rng.normal(0, 0.3, orc.mlp_nparams())
    return P


def _numpy_forward(X, P):
    H, F = 64, 8
    o = 0
    W1 = P[o:o + H * F].reshape(H, F); o += H * F
    b1 = P[o:o + H]; o += H
    W2 = P[o:o + H * H].reshape(H, H); o += H * H
    b2 = P[o:o + H]; o += H
    W3 = P[o:o + H * H].reshape(H, H); o += H * H
    b3 = P[o:o + H]; o += H
    W4 = P[o:o + H]; o += H
    b4 = P[o]
    silu = lambda z: z / (1 + np.exp(-z))
    h = silu(X @ W1.T + b1)
    h = silu(h @ W2.T + b2)
    h = silu(h @ W3.T + b3)
    return h @ W4 + b4


def test_forward_matches_numpy(orc):
    rng = np.random.default_rng(0)
    X = rng.normal(0, 1, (50, 8))
    P = _params(rng, orc)
    assert np.allclose(orc.mlp_forward(X, P), _numpy_forward(X, P), rtol=1e-12, atol=1e-12)


def test_gradient_finite_differences(orc):
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (20, 8))
    t = rng.normal(0, 1, 20)
    P = _params(rng, orc)
    loss, G = orc.mlp_loss_grad(X, t, P)
    assert abs(loss - np.mean((_numpy_forward(X, P) - t) ** 2)) <= 1e-12 * loss
    idx = rng.choice(len(P), 60, replace=False)
    idx = np.concatenate([idx, [len(P) - 1, len(P) - 2, 0, 64 * 8]])  # b4, W4, W1, b1
    for k in idx:
        e = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += e
        Pm[k] -= e
        fd = (orc.mlp_loss_grad(X, t, Pp)[0] - orc.mlp_loss_grad(X, t, Pm)[0]) / (2 * e)
        assert abs(fd - G[k]) <= 1e-6 * max(1.0, abs(G[k])), (k, fd, G[k])
