"""FP64 CPU reference of the warm-start MLP (test infrastructure only).

Plain numpy, written from the definition of the network and of the mean
squared error, independent of the CUDA kernels:

    A1 = tanh(X W1^T + b1),  A2 = tanh(A1 W2^T + b2),  Y = A2 W3^T + b3,
    loss = mean((Y - T)^2) over all samples and outputs.

The flat parameter vector is [W1 (nh x nin, row-major), b1, W2 (nh x nh),
b2, W3 (nout x nh), b3]; the gradient uses the same layout.
"""
from __future__ import annotations

import numpy as np


def unpack(theta, nin, nh, nout):
    theta = np.asarray(theta, dtype=np.float64)
    k = 0
    W1 = theta[k:k + nh * nin].reshape(nh, nin); k += nh * nin
    b1 = theta[k:k + nh]; k += nh
    W2 = theta[k:k + nh * nh].reshape(nh, nh); k += nh * nh
    b2 = theta[k:k + nh]; k += nh
    W3 = theta[k:k + nout * nh].reshape(nout, nh); k += nout * nh
    b3 = theta[k:k + nout]; k += nout
    assert k == theta.size
    return W1, b1, W2, b2, W3, b3


def size(nin, nh, nout):
    return nh * nin + nh + nh * nh + nh + nout * nh + nout


def forward(theta, X, nin, nh, nout):
    W1, b1, W2, b2, W3, b3 = unpack(theta, nin, nh, nout)
    A1 = np.tanh(X @ W1.T + b1)
    A2 = np.tanh(A1 @ W2.T + b2)
    return A2 @ W3.T + b3, (A1, A2)


def loss(theta, X, T, nin, nh, nout):
    Y, _ = forward(theta, X, nin, nh, nout)
    return float(np.mean((Y - T) ** 2))


def loss_grad(theta, X, T, nin, nh, nout):
    """(loss, gradient) by the chain rule, layer by layer."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(theta, nin, nh, nout)
    Y, (A1, A2) = forward(theta, X, nin, nh, nout)
    D = Y - T
    L = float(np.mean(D ** 2))
    dY = 2.0 * D / D.size
    dW3 = dY.T @ A2
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3) * (1.0 - A2 ** 2)
    dW2 = dZ2.T @ A1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (1.0 - A1 ** 2)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, g
