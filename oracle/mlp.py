"""FP64 reference of the learned residual correction (MLP + features + Adam).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and never imports it.

The paper maps the aperture mass two ways, galaxy by galaxy (Sect. 3.1)
and from pixel-binned shear (Sect. 3.2); the second is much cheaper but
moves every galaxy to its pixel centre.  The learned part predicts, per
output pixel, the difference M_bf^E - M_pix^E between the two maps from four
per-pixel features of the pixel-based map:

    f = [ M_pix^E,  sum_w,  var(n_p over the aperture's pixels),  z ]

where var(n_p) = sum n_p^2 / K - (sum n_p / K)^2 over the K pixels whose
centres lie in the aperture (the membership of Sect. 3.2, fourth step) and
z = cos(colatitude) of the output pixel centre.  Features and target are
standardised with the training set's mean and population standard
deviation.  The network is 4 -> 64 -> 64 -> 1 with SiLU activations,
trained on the mean squared error with Adam (Kingma & Ba 2015): the
architecture, loss and optimiser are this library's reading, the paper
prescribes none of them.

Parameter vector layout (float32 master copy, also the library's):
    W1 [64][4], b1 [64], W2 [64][64], b2 [64], w3 [64], b3  -> 4545 values
with W[out][in] row-major.  In "bf16" mode the weight matrices W1, W2, w3
take their bfloat16-rounded values (round to nearest, ties to even); the
biases stay float32.

Everything here is float64 numpy.  ``act="bf16"`` additionally rounds the
two tensor-core operands the library rounds (the first hidden activation
and the gradient at the second pre-activation) to bfloat16, so that a test
can compare the library's arithmetic order-for-order.
"""
from __future__ import annotations

import numpy as np

from . import query_disc

F = 4
H = 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAMS = OFF_B3 + 1
WEIGHT_BLOCKS = ((OFF_W1, H * F), (OFF_W2, H * H), (OFF_W3, H))


# --------------------------------------------------------------------------
# features (Sect. 3.2 membership) and standardisation
# --------------------------------------------------------------------------
def disc_count_moments(nside_bin: int, centres, n_p, theta_ap: float):
    """(K, sum n_p, sum n_p^2) over the binned pixels whose centre lies within
    theta_ap of each centre (exact float64 membership, Sect. 3.2)."""
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    n_p = np.asarray(n_p, np.int64)
    K = np.zeros(len(centres), np.int64)
    S1 = np.zeros(len(centres), np.int64)
    S2 = np.zeros(len(centres), np.int64)
    for t, r0 in enumerate(centres):
        pix = query_disc(nside_bin, r0, theta_ap)
        c = n_p[pix]
        K[t] = pix.size
        S1[t] = int(c.sum())
        S2[t] = int((c * c).sum())
    return K, S1, S2


def features(map_e, sum_w, count, members, sum_n2, z) -> np.ndarray:
    """Raw feature rows [M_pix^E, sum_w, var(n_p), z] (float64, shape (n, 4))."""
    K = np.asarray(members, np.float64)
    mean_n = np.divide(np.asarray(count, np.float64), K, out=np.zeros_like(K), where=K > 0)
    mean_n2 = np.divide(np.asarray(sum_n2, np.float64), K, out=np.zeros_like(K), where=K > 0)
    return np.stack([np.asarray(map_e, np.float64), np.asarray(sum_w, np.float64),
                     mean_n2 - mean_n * mean_n, np.asarray(z, np.float64)], axis=1)


def fit_scaler(feat, target):
    """Mean and population standard deviation of each feature and of the target."""
    feat = np.asarray(feat, np.float64)
    target = np.asarray(target, np.float64)
    mu = feat.mean(axis=0)
    sd = feat.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    t_sd = target.std()
    return mu, sd, float(target.mean()), float(t_sd if t_sd > 0 else 1.0)


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of the float32 encoding; rounding adds
    0x7FFF plus the lowest kept bit before truncating (finite inputs)."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta, weights: str = "bf16") -> dict:
    th = np.asarray(theta, np.float64)
    assert th.size == NPARAMS
    p = {"W1": th[OFF_W1:OFF_B1].reshape(H, F), "b1": th[OFF_B1:OFF_W2],
         "W2": th[OFF_W2:OFF_B2].reshape(H, H), "b2": th[OFF_B2:OFF_W3],
         "w3": th[OFF_W3:OFF_B3], "b3": th[OFF_B3]}
    if weights == "bf16":
        for k in ("W1", "W2", "w3"):
            p[k] = bf16_round(p[k])
    return p


def silu(a):
    return a / (1.0 + np.exp(-a))


def dsilu(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def forward(theta, X, weights: str = "bf16", act: str = "exact"):
    """y (n,) for standardised inputs X (n, 4), and the cache for backward."""
    p = unpack(theta, weights)
    X = np.asarray(X, np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = silu(a1)
    if act == "bf16":
        h1 = bf16_round(h1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(a2)
    y = h2 @ p["w3"] + p["b3"]
    return y, dict(p=p, X=X, a1=a1, h1=h1, a2=a2, h2=h2)


def loss_and_grad(theta, X, t, weights: str = "bf16", act: str = "exact"):
    """L = mean((y - t)^2) and dL/dtheta (flat, NPARAMS).

    In bf16 mode the gradient is taken with respect to the rounded weights
    (the straight-through convention: the float32 master copy receives it)."""
    y, c = forward(theta, X, weights, act)
    p = c["p"]
    n = y.size
    d = y - np.asarray(t, np.float64)
    L = float(np.mean(d * d))
    dy = 2.0 * d / n
    g = np.zeros(NPARAMS)
    g[OFF_W3:OFF_B3] = c["h2"].T @ dy
    g[OFF_B3] = dy.sum()
    da2 = np.outer(dy, p["w3"]) * dsilu(c["a2"])
    g[OFF_B2:OFF_W3] = da2.sum(axis=0)
    da2_op = bf16_round(da2) if act == "bf16" else da2
    g[OFF_W2:OFF_B2] = (da2_op.T @ c["h1"]).ravel()
    dh1 = da2_op @ p["W2"]
    da1 = dh1 * dsilu(c["a1"])
    g[OFF_W1:OFF_B1] = (da1.T @ c["X"]).ravel()
    g[OFF_B1:OFF_W2] = da1.sum(axis=0)
    return L, g


# --------------------------------------------------------------------------
# optimiser (Kingma & Ba 2015, Algorithm 1)
# --------------------------------------------------------------------------
def adam_step(theta, m, v, g, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step number ``step`` (1-based); returns (theta, m, v)."""
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return np.asarray(theta, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def train(theta, X, t, batches, lr: float, weights: str = "bf16", act: str = "exact"):
    """Adam over the given minibatches (lists of row indices); returns
    (theta, m, v, losses)."""
    theta = np.asarray(theta, np.float64).copy()
    m = np.zeros(NPARAMS)
    v = np.zeros(NPARAMS)
    losses = []
    for k, idx in enumerate(batches, start=1):
        L, g = loss_and_grad(theta, X[idx], t[idx], weights, act)
        theta, m, v = adam_step(theta, m, v, g, k, lr)
        losses.append(L)
    return theta, m, v, losses
