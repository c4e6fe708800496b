"""FP64 oracle of the learned initial guess (features, MLP, loss, gradient).

Test infrastructure only (see ``oracle/__init__``).

Features of a scatterer (448 values, by their definition): for each of the
48 lattice offsets (dx, dy) with 0 < dx^2 + dy^2 <= 16 cells (2 wavelengths
at pitch 0.5), ordered by dx^2 + dy^2 and then by atan2(dy, dx): a one-hot
shape id (8) and a presence flag (1) of the neighbour at that offset in the
same array; then the scatterer's own shape one-hot (8), the incidence
direction (3), the real part of the polarisation (3) and two zeros.

Network: 4 dense layers dims[0] -> dims[1] -> dims[2] -> dims[3] -> dims[4],
SiLU after the first three, y = x W + b with W stored [in][out]; parameters
flat, layer by layer, W then b.  Loss: mean of squared errors over all
outputs.  Gradient by backpropagation (checked against central differences
in the tests).
"""
import math

import numpy as np


def slots():
    out = []
    for dy in range(-4, 5):
        for dx in range(-4, 5):
            d2 = dx * dx + dy * dy
            if 0 < d2 <= 16:
                out.append((d2, math.atan2(dy, dx), dx, dy))
    out.sort()
    return [(dx, dy) for (_, _, dx, dy) in out]


def lattice_indices(centres, array_ids, pitch):
    """Integer lattice index of each particle in its own array's frame."""
    C = np.asarray(centres, dtype=float)
    A = np.asarray(array_ids)
    ij = np.zeros((len(C), 2), dtype=int)
    for a in np.unique(A):
        sel = A == a
        o = C[sel, :2].min(axis=0)
        ij[sel] = np.rint((C[sel, :2] - o) / pitch).astype(int)
    return ij


def features(centres, shape_ids, array_ids, khat, pol, pitch=0.5):
    """(p, 448) features; khat (n_arrays, 3), pol (n_arrays, 3) complex."""
    ij = lattice_indices(centres, array_ids, pitch)
    S = np.asarray(shape_ids)
    A = np.asarray(array_ids)
    where = {(int(A[i]), int(ij[i, 0]), int(ij[i, 1])): i for i in range(len(S))}
    sl = slots()
    F = np.zeros((len(S), 448))
    for i in range(len(S)):
        for s, (dx, dy) in enumerate(sl):
            nu = where.get((int(A[i]), int(ij[i, 0]) + dx, int(ij[i, 1]) + dy))
            if nu is not None:
                F[i, 9 * s + S[nu]] = 1.0
                F[i, 9 * s + 8] = 1.0
        F[i, 432 + S[i]] = 1.0
        F[i, 440:443] = np.asarray(khat, dtype=float)[A[i]]
        F[i, 443:446] = np.real(np.asarray(pol)[A[i]])
    return F


def unpack(params, dims):
    p = np.asarray(params, dtype=float)
    out, o = [], 0
    for l in range(4):
        n_in, n_out = dims[l], dims[l + 1]
        W = p[o:o + n_in * n_out].reshape(n_in, n_out)
        o += n_in * n_out
        b = p[o:o + n_out]
        o += n_out
        out.append((W, b))
    assert o == p.size
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, dims, X):
    layers = unpack(params, dims)
    A = np.asarray(X, dtype=float)
    cache = [A]
    for l, (W, b) in enumerate(layers):
        Z = A @ W + b
        A = silu(Z) if l < 3 else Z
        cache.append(Z)
        if l < 3:
            cache.append(A)
    return A, cache


def loss_grad(params, dims, X, T):
    """(loss, flat gradient) of mean((Y - T)^2)."""
    Y, cache = forward(params, dims, X)
    T = np.asarray(T, dtype=float)
    n, O = Y.shape
    loss = float(np.mean((Y - T) ** 2))
    dZ = 2.0 * (Y - T) / (n * O)
    layers = unpack(params, dims)
    grads = [None] * 4
    # cache: [X, Z1, A1, Z2, A2, Z3, A3, Z4]
    acts = [cache[0], cache[2], cache[4], cache[6]]
    zs = [cache[1], cache[3], cache[5], cache[7]]
    for l in range(3, -1, -1):
        W, _ = layers[l]
        gW = acts[l].T @ dZ
        gb = dZ.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dZ = (dZ @ W.T) * dsilu(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
