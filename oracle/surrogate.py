"""FP64 reference of the learned surrogate (test infrastructure, see oracle/__init__).

The paper has no surrogate; this is the CPU definition that the GPU training
and inference kernels are checked against.  The network maps an 8-feature
description of a macro Gauss point to the Cholesky factors of its normalised
homogenised tensors, so every prediction is symmetric positive definite:

    h_0 = x,  h_{l+1} = silu(h_l W_l + b_l)  (l = 0..3, width 256),
    z = h_4 W_4 + b_4  (33 outputs),
    L = tril(z) with softplus on the diagonal entries, C = L L^T (21 + 6 + 6).

Loss: mean over samples and outputs of ((L(z) - L_target) / sigma)^2, sigma a
fixed per-output scale.  Pinned by central finite differences (gradients) and
by the SPD property of every reconstruction (tests/test_oracle_surrogate.py).
"""
from __future__ import annotations

import numpy as np

WIDTH = 256
DEPTH = 4
N_IN = 8
N_OUT = 33          # 21 (6x6) + 6 (3x3) + 6 (3x3) lower-triangular entries
BLOCKS = ((6, 0), (3, 21), (3, 27))   # (size, offset) of each tensor's factor


def tril_indices(n):
    """Row-major lower triangle: (0,0), (1,0), (1,1), (2,0), ..."""
    return [(i, j) for i in range(n) for j in range(i + 1)]


def diagonal_mask():
    m = np.zeros(N_OUT, bool)
    for n, off in BLOCKS:
        for k, (i, j) in enumerate(tril_indices(n)):
            m[off + k] = i == j
    return m


DIAG = diagonal_mask()


def silu(a):
    return a / (1.0 + np.exp(-a))


def dsilu(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def softplus(a):
    return np.logaddexp(0.0, a)


def init_params(seed, width=WIDTH, depth=DEPTH, n_in=N_IN, n_out=N_OUT):
    """He-style uniform initialisation; list of (W [in,out], b [out])."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * depth + [n_out]
    params = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = np.sqrt(6.0 / a)
        params.append((rng.uniform(-lim, lim, size=(a, b)), np.zeros(b)))
    return params


def forward(params, x):
    """Returns z [B,33] and the cache of pre-activations for backward."""
    h = np.asarray(x, float)
    cache = []
    for l, (W, b) in enumerate(params):
        a = h @ W + b
        cache.append((h, a))
        h = silu(a) if l < len(params) - 1 else a
    return h, cache


def factor_entries(z):
    """Cholesky-factor entries from raw outputs (softplus on diagonals)."""
    return np.where(DIAG, softplus(z), z)


def tensors_from_factors(Lv):
    """[B,33] factor entries -> (C [B,6,6], K [B,3,3], D [B,3,3]) = L L^T."""
    out = []
    for n, off in BLOCKS:
        L = np.zeros((Lv.shape[0], n, n))
        for k, (i, j) in enumerate(tril_indices(n)):
            L[:, i, j] = Lv[:, off + k]
        out.append(np.einsum("bij,bkj->bik", L, L))
    return out


def factors_from_tensors(C, K, D):
    """Inverse of tensors_from_factors via the Cholesky decomposition."""
    B = C.shape[0]
    Lv = np.zeros((B, N_OUT))
    for T, (n, off) in zip((C, K, D), BLOCKS):
        L = np.linalg.cholesky(T)
        for k, (i, j) in enumerate(tril_indices(n)):
            Lv[:, off + k] = L[:, i, j]
    return Lv


def loss_and_grads(params, x, target, sigma):
    """Mean squared error of the factor entries and its parameter gradients."""
    z, cache = forward(params, x)
    Lv = factor_entries(z)
    B = x.shape[0]
    r = (Lv - target) / sigma
    loss = float(np.mean(r ** 2))
    dL = 2.0 * r / sigma / (B * N_OUT)
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = np.where(DIAG, dL * sig, dL)
    grads = [None] * len(params)
    g = dz
    for l in range(len(params) - 1, -1, -1):
        h, a = cache[l]
        W, _ = params[l]
        grads[l] = (h.T @ g, g.sum(axis=0))
        if l > 0:
            _, a_prev = cache[l - 1]
            g = (g @ W.T) * dsilu(a_prev)
    return loss, grads


def adam_step(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); state is a list of (m_W, v_W, m_b, v_b)."""
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        mW, vW, mb, vb = state[l]
        mW = b1 * mW + (1 - b1) * gW
        vW = b2 * vW + (1 - b2) * gW * gW
        mb = b1 * mb + (1 - b1) * gb
        vb = b2 * vb + (1 - b2) * gb * gb
        c1, c2 = 1 - b1 ** t, 1 - b2 ** t
        W = W - lr * (mW / c1) / (np.sqrt(vW / c2) + eps)
        b = b - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)
        state[l] = (mW, vW, mb, vb)
        out.append((W, b))
    return out
