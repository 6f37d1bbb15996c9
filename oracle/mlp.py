"""FP64 reference of the learned-initial-guess network (TEST INFRASTRUCTURE ONLY).

Plain numpy: standardise the inputs, dense layers with GELU (erf form) on the
hidden layers, mean-squared error, gradients by hand-written backpropagation.
The parameter vector layout is the library's: layer by layer W [out][in] then
b [out], then the input means and inverse standard deviations.  Used only to
check the CUDA training kernels; pinned by central finite differences.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def layer_dims(nin: int, hidden: int, nhidden: int, nout: int):
    dims = [nin] + [hidden] * nhidden + [nout]
    return list(zip(dims[:-1], dims[1:]))


def unpack(state, nin, hidden, nhidden, nout):
    state = np.asarray(state, dtype=np.float64)
    off = 0
    Ws, bs = [], []
    for di, do in layer_dims(nin, hidden, nhidden, nout):
        Ws.append(state[off:off + di * do].reshape(do, di))
        off += di * do
        bs.append(state[off:off + do])
        off += do
    mean = state[off:off + nin]
    istd = state[off + nin:off + 2 * nin]
    return Ws, bs, mean, istd, off


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(state, dims4, X):
    Ws, bs, mean, istd, _ = unpack(state, *dims4)
    h = (np.asarray(X, dtype=np.float64) - mean) * istd
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        h = gelu(z) if l < len(Ws) - 1 else z
    return h


def loss_grad(state, dims4, X, Y):
    """Mean squared error over all rows and outputs and its gradient with
    respect to the weights and biases (zeros for the standardisation)."""
    Ws, bs, mean, istd, nwb = unpack(state, *dims4)
    h = (np.asarray(X, dtype=np.float64) - mean) * istd
    hs, zs = [h], []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        zs.append(z)
        h = gelu(z) if l < len(Ws) - 1 else z
        hs.append(h)
    pred = h
    d = pred - np.asarray(Y, dtype=np.float64)
    loss = float(np.mean(d * d))
    dz = 2.0 * d / d.size
    grads = []
    for l in range(len(Ws) - 1, -1, -1):
        gW = dz.T @ hs[l]
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            dz = (dz @ Ws[l]) * gelu_grad(zs[l - 1])
    grads.reverse()
    g = np.zeros(len(np.asarray(state)))
    off = 0
    for gW, gb in grads:
        g[off:off + gW.size] = gW.reshape(-1)
        off += gW.size
        g[off:off + gb.size] = gb
        off += gb.size
    return loss, g


def features(T, ne, nH, vz):
    """[T | log10 n_e | log10 n_H | v_z] per depth, per column."""
    return np.concatenate([T, np.log10(ne), np.log10(nH), vz], axis=1)
