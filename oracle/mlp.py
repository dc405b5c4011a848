"""Plain FP64 numpy reference of the learned-culling network -- TEST INFRASTRUCTURE.

The network of the library's learned culling: x -> (x - mu) * inv_sigma ->
three dense layers of width 64 with the exact GELU, 0.5 z (1 + erf(z/sqrt 2)),
-> one linear output.  Loss 0.5 * mean((y - t)^2).  Parameter vector layout
(float): mu[10], inv_sigma[10], W1[64][10], b1[64], W2[64][64], b2[64],
W3[64][64], b3[64], W4[64], b4.  The normalisation vectors are not trained.

Forward, analytic backward and one Adam step, written out so that a reader
can check them line by line; the analytic gradient is pinned by central
finite differences in tests/test_oracle_mlp.py.  Nothing here is used by the
library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

NF, NH = 10, 64
P_MU, P_IS, P_W1 = 0, NF, 2 * NF
P_B1 = P_W1 + NH * NF
P_W2 = P_B1 + NH
P_B2 = P_W2 + NH * NH
P_W3 = P_B2 + NH
P_B3 = P_W3 + NH * NH
P_W4 = P_B3 + NH
P_B4 = P_W4 + NH
NP = P_B4 + 1


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return dict(mu=p[P_MU:P_IS], isg=p[P_IS:P_W1], W1=p[P_W1:P_B1].reshape(NH, NF), b1=p[P_B1:P_W2],
                W2=p[P_W2:P_B2].reshape(NH, NH), b2=p[P_B2:P_W3], W3=p[P_W3:P_B3].reshape(NH, NH),
                b3=p[P_B3:P_W4], W4=p[P_W4:P_B4], b4=p[P_B4])


def forward(p, X):
    q = unpack(p)
    a0 = (np.asarray(X, np.float64) - q["mu"]) * q["isg"]
    z1 = a0 @ q["W1"].T + q["b1"]
    a1 = gelu(z1)
    z2 = a1 @ q["W2"].T + q["b2"]
    a2 = gelu(z2)
    z3 = a2 @ q["W3"].T + q["b3"]
    a3 = gelu(z3)
    y = a3 @ q["W4"] + q["b4"]
    return y, (a0, z1, a1, z2, a2, z3, a3)


def loss_grad(p, X, T):
    """Loss 0.5 * mean((y - T)^2) and its gradient (zero for mu, inv_sigma)."""
    q = unpack(p)
    y, (a0, z1, a1, z2, a2, z3, a3) = forward(p, X)
    n = y.shape[0]
    e = y - np.asarray(T, np.float64)
    loss = 0.5 * np.mean(e * e)
    dy = e / n
    g = np.zeros(NP)
    g[P_W4:P_B4] = a3.T @ dy
    g[P_B4] = dy.sum()
    d3 = np.outer(dy, q["W4"]) * gelu_d(z3)
    g[P_W3:P_B3] = (d3.T @ a2).ravel()
    g[P_B3:P_W4] = d3.sum(0)
    d2 = (d3 @ q["W3"]) * gelu_d(z2)
    g[P_W2:P_B2] = (d2.T @ a1).ravel()
    g[P_B2:P_W3] = d2.sum(0)
    d1 = (d2 @ q["W2"]) * gelu_d(z1)
    g[P_W1:P_B1] = (d1.T @ a0).ravel()
    g[P_B1:P_W2] = d1.sum(0)
    return loss, g


def adam(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step on the trained parameters."""
    p, m, v = p.copy(), m.copy(), v.copy()
    sl = slice(P_W1, NP)
    m[sl] = b1 * m[sl] + (1 - b1) * g[sl]
    v[sl] = b2 * v[sl] + (1 - b2) * g[sl] ** 2
    mh = m[sl] / (1 - b1 ** step)
    vh = v[sl] / (1 - b2 ** step)
    p[sl] = p[sl] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
