"""FP64 oracle of the learned angular decimation -- test infrastructure only.

Sec. 2.1 leaves the angular low-pass of the decomposition open and says
its implementation sets the quality.  The learned form replaces the plain
low-pass by the plain one plus a small residual network along the view
axis.  For each detector row v and shifted column t of a square, the input
is that column's shifted sequence x[k] = S_q[k][v][t] over all P views
(circular: the orbit is closed), and, with C = 16 channels and K = 5 taps
at offsets m - 2, m = 0 .. 4 (cross-correlation):

    z1[c][k] = sum_m W1[c][m] x[k + m - 2],                a1 = max(z1, 0)
    z2[c][k] = sum_{c', m} W2[c][c'][m] a1[c'][k + m - 2],  a2 = max(z2, 0)
    y[j]     = sum_{c, m} W3[c][m] a2[c][j D + m - 2]       (stride D)

and the decimated view is S'_q[j][v][t] = (plain low-pass, every D-th view)
+ y[j].  No biases: the net is positively homogeneous, so scaling a scan
scales its reconstruction, as the rest of FDK does.

The weights travel as one flat vector (the layout of the C interface):
W1 [C][K], then W2 [C][C][K] (output channel, input channel, tap), then
W3 [C][K]; NET_SIZE = 1440 values.

Functions:
  net_unpack / net_pack        flat vector <-> (W1, W2, W3)
  net_forward(x, D, w)         y for a batch of sequences x[P][...]
  net_vjp(x, D, w, dy)         gradient of sum(dy * y) with respect to w
  net_loop(x, D, w)            the same forward with explicit loops (tiny
                               inputs; an independent restatement for pins)
  round_bf16, act_rounding_bound  BF16 storage of the layers' inputs (the
                               tensor-core operands) and a bound on what it changes
Pins in tests/test_oracle_net.py.
"""
from __future__ import annotations

import numpy as np

C = 16
K = 5
NET_SIZE = C * K + C * C * K + C * K


def net_unpack(w):
    w = np.asarray(w, dtype=np.float64).reshape(-1)
    if w.size != NET_SIZE:
        raise ValueError(f"net weights hold {NET_SIZE} values")
    W1 = w[:C * K].reshape(C, K)
    W2 = w[C * K:C * K + C * C * K].reshape(C, C, K)
    W3 = w[C * K + C * C * K:].reshape(C, K)
    return W1, W2, W3


def net_pack(W1, W2, W3) -> np.ndarray:
    return np.concatenate([np.asarray(W1, np.float64).reshape(-1), np.asarray(W2, np.float64).reshape(-1),
                           np.asarray(W3, np.float64).reshape(-1)])


def _ahead(a, d):
    """a[k + d] along axis 1 (the view axis of [channel][view][...]),
    circular."""
    return np.roll(a, -d, axis=1)


def round_bf16(a):
    """Nearest value with an 8-bit significand (BF16), ties to even,
    computed exactly in FP64 (normal range)."""
    a = np.asarray(a, dtype=np.float64)
    _, e = np.frexp(a)                                  # a = f 2^e, 0.5 <= |f| < 1
    scale = np.ldexp(1.0, e - 8)
    return np.round(a / scale) * scale


def _layers(x, w, act_round=None):
    """x, z1, a1, z2, a2, W3; act_round="bf16" rounds every layer's input
    (x, a1, a2) to BF16, the operands of a tensor-core evaluation."""
    if act_round not in (None, "bf16"):
        raise ValueError(f"unknown act_round {act_round!r}")
    rnd = round_bf16 if act_round == "bf16" else (lambda a: a)
    W1, W2, W3 = net_unpack(w)
    x = rnd(np.asarray(x, dtype=np.float64)[None])     # [1][P][...]
    z1 = sum(W1[:, m].reshape((C, 1) + (1,) * (x.ndim - 2)) * _ahead(x, m - 2) for m in range(K))
    a1 = rnd(np.maximum(z1, 0.0))
    z2 = np.zeros_like(a1)
    for m in range(K):
        z2 += np.tensordot(W2[:, :, m], _ahead(a1, m - 2), axes=(1, 0))
    a2 = rnd(np.maximum(z2, 0.0))
    return x, z1, a1, z2, a2, W3


def net_forward(x, D: int, w, act_round=None) -> np.ndarray:
    """y[j][...] for sequences x[P][...] (P divisible by D).  act_round="bf16"
    rounds x, a1 and a2 to BF16 (the tensor-core operands) before the layer
    that reads them."""
    x, _, _, _, a2, W3 = _layers(x, w, act_round)
    P = x.shape[1]
    if P % D:
        raise ValueError("D must divide P")
    full = sum(np.tensordot(W3[:, m], _ahead(a2, m - 2), axes=(0, 0)) for m in range(K))
    return full[::D]


def net_vjp(x, D: int, w, dy) -> np.ndarray:
    """Flat gradient of sum(dy * net_forward(x, D, w)) with respect to w
    (ReLU derivative 0 at 0)."""
    x, z1, a1, z2, a2, W3 = _layers(x, w)
    _, W2, _ = net_unpack(w)
    dfull = np.zeros(x.shape[1:])
    dfull[::D] = np.asarray(dy, dtype=np.float64)
    red = tuple(range(1, x.ndim))                      # sum over views and batch
    # layer 3: full[k] = sum_{c,m} W3[c][m] a2[c][k + m - 2]
    dW3 = np.stack([(a2 * _ahead(dfull[None], -(m - 2))).sum(axis=red) for m in range(K)], axis=1)
    da2 = sum(W3[:, m].reshape((C, 1) + (1,) * (x.ndim - 2)) * _ahead(dfull[None], -(m - 2)) for m in range(K))
    dz2 = da2 * (z2 > 0)
    # layer 2: z2[c][k] = sum_{c',m} W2[c][c'][m] a1[c'][k + m - 2]
    dW2 = np.stack([np.tensordot(dz2, _ahead(a1, m - 2), axes=(red, red)) for m in range(K)], axis=2)
    da1 = np.zeros_like(a1)
    for m in range(K):
        da1 += np.tensordot(W2[:, :, m], _ahead(dz2, -(m - 2)), axes=(0, 0))
    dz1 = da1 * (z1 > 0)
    # layer 1: z1[c][k] = sum_m W1[c][m] x[k + m - 2]
    dW1 = np.stack([(dz1 * _ahead(x, m - 2)).sum(axis=red) for m in range(K)], axis=1)
    return net_pack(dW1, dW2, dW3)


def net_loop(x, D: int, w) -> np.ndarray:
    """net_forward for x[P][B] by explicit loops over every index (slow;
    for tiny P and B only)."""
    W1, W2, W3 = net_unpack(w)
    x = np.asarray(x, dtype=np.float64)
    P, B = x.shape
    y = np.zeros((P // D, B))
    for b in range(B):
        a1 = [[0.0] * P for _ in range(C)]
        for c in range(C):
            for k in range(P):
                acc = 0.0
                for m in range(K):
                    acc += W1[c][m] * x[(k + m - 2) % P][b]
                a1[c][k] = acc if acc > 0.0 else 0.0
        a2 = [[0.0] * P for _ in range(C)]
        for c in range(C):
            for k in range(P):
                acc = 0.0
                for ci in range(C):
                    for m in range(K):
                        acc += W2[c][ci][m] * a1[ci][(k + m - 2) % P]
                a2[c][k] = acc if acc > 0.0 else 0.0
        for j in range(P // D):
            acc = 0.0
            for c in range(C):
                for m in range(K):
                    acc += W3[c][m] * a2[c][(j * D + m - 2) % P]
            y[j][b] = acc
    return y


def linear_net(g3, offsets=(1, -2), chans=(3, 11, 5, 9)) -> np.ndarray:
    """Weights under which the net is linear: channel pair (ca, cb) of layer
    1 carries relu(x[k + o1]) and relu(-x[k + o1]); pair (cc, cd) of layer 2
    carries relu(+-x[k + o1 + o2]); layer 3 gives y[j] = sum_m g3[m]
    x[j D + m - 2 + o1 + o2].  Used to pin the net's indexing against the
    plain linear low-pass (relu(u) - relu(-u) = u)."""
    o1, o2 = offsets
    ca, cb, cc, cd = chans
    W1 = np.zeros((C, K))
    W2 = np.zeros((C, C, K))
    W3 = np.zeros((C, K))
    W1[ca, o1 + 2] = 1.0
    W1[cb, o1 + 2] = -1.0
    W2[cc, ca, o2 + 2] = 1.0
    W2[cc, cb, o2 + 2] = -1.0
    W2[cd, cb, o2 + 2] = 1.0
    W2[cd, ca, o2 + 2] = -1.0
    W3[cc, :] = g3
    W3[cd, :] = -np.asarray(g3, np.float64)
    return net_pack(W1, W2, W3)


def act_rounding_bound(x, D: int, w, u: float = 2.0 ** -8) -> np.ndarray:
    """Elementwise bound, to first order in u, on the change of
    net_forward(x, D, w) when every x, a1 and a2 value is rounded with
    relative error at most u (storage of unit roundoff u): ReLU is
    1-Lipschitz and each layer is linear in its input, so the change is at
    most u (|W3| |a2| + |W3| |W2| |a1| + |W3| |W2| |W1| |x|) at the output
    positions, |W| the layers with absolute weights; the factor 1 + 4u
    absorbs the higher-order terms."""
    x, _, a1, _, a2, _ = _layers(x, w)
    W1, W2, W3 = net_unpack(w)
    ax = np.abs(x)
    e1 = sum(np.abs(W1[:, m]).reshape((C, 1) + (1,) * (ax.ndim - 2)) * _ahead(ax, m - 2) for m in range(K))
    e2 = np.zeros_like(a1)
    for m in range(K):
        e2 += np.tensordot(np.abs(W2[:, :, m]), _ahead(a1 + e1, m - 2), axes=(1, 0))
    e3 = a2 + e2
    full = sum(np.tensordot(np.abs(W3[:, m]), _ahead(e3, m - 2), axes=(0, 0)) for m in range(K))
    return u * (1.0 + 4.0 * u) * full[::D]
