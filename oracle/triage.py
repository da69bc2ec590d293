"""Plain FP64 CPU oracle of the learned sky triage.

THIS MODULE IS TEST INFRASTRUCTURE, like the rest of ``oracle/``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
use it, and it shares no code with the CUDA library.

The paper has no learned component; the triage ranks sky patches for the
exhaustive search of Sec. 2 / Eq. 4 and is defined here from scratch:

  sky_order       the sky sorted by its Doppler factor v_0(t_m).nhat (Eq. 2),
                  t_m = middle segment of detector 0, ties by sky index
  patches         patch p = sorted positions [p P, min((p + 1) P, S));
                  representative = sorted position p P + (len - 1) // 2
  coarse_psi      Psi of Eq. 4 for every template at every representative,
                  from the FP64 oracle's search_stats
  histogram_features
                  per patch, the histogram of those Psi over 128 equal bins
                  of [lo, hi) (values below lo and -inf in bin 0, values at
                  or above hi in bin 127); feature = log(1 + count)
  mlp_forward     128 -> 256 -> 256 -> 1 with ReLU after the two hidden
                  layers; weights rounded to bfloat16, arithmetic in FP64
  mlp_backward    gradients of a scalar loss by the chain rule
  bce_with_logits mean binary cross-entropy with logits (positive weight pw)
                  and its derivative
  adam_step       Adam with bias correction

Packed parameter layout (float64 here, float32 masters on the GPU):
  W1 [128][256], b1 [256], W2 [256][256], b2 [256], w3 [256], b3 [1]
  y = relu(relu(X W1 + b1) W2 + b2) w3 + b3
"""
from __future__ import annotations

import numpy as np

from . import search_stats

N_IN, N_H1, N_H2 = 128, 256, 256
SIZES = [("W1", (N_IN, N_H1)), ("b1", (N_H1,)), ("W2", (N_H1, N_H2)), ("b2", (N_H2,)),
         ("w3", (N_H2,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    """Views of the packed parameter vector, by name."""
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n]).reshape(shape)
        off += n
    return out


def bf16_round(x):
    """Round float32(x) to the nearest bfloat16 (ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    r = np.where(nan, u, r).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def sky_order(velocity, nhat):
    """Sorted sky indices by v_0(t_m).nhat, t_m = the middle segment."""
    v = np.asarray(velocity, np.float64)[0, v_mid_index(velocity)]
    n = np.asarray(nhat, np.float64)
    key = v[0] * n[:, 0] + v[1] * n[:, 1] + v[2] * n[:, 2]
    return np.argsort(key, kind="stable")


def v_mid_index(velocity):
    return np.asarray(velocity).shape[1] // 2


def patches(n_sky, patch_size):
    """(first sorted position, length, representative sorted position) per patch."""
    out = []
    for p0 in range(0, n_sky, patch_size):
        ln = min(patch_size, n_sky - p0)
        out.append((p0, ln, p0 + (ln - 1) // 2))
    return out


def coarse_psi(rho, f_min, df, t_mid, weights, velocity, nhat, f0, tau, n, T0, patch_size):
    """Psi [n_patch][B] at each patch's representative sky (FP64 oracle)."""
    order = sky_order(velocity, nhat)
    reps = [order[r] for _, _, r in patches(len(order), patch_size)]
    _, _, _, psi = search_stats(rho, f_min, df, t_mid, weights, velocity,
                                np.asarray(nhat, np.float64)[reps], f0, tau, n, T0)
    return psi


def histogram_features(psi, lo, hi, n_bins=N_IN):
    """Counts of each row of psi in n_bins equal bins of [lo, hi) and log1p(counts)."""
    psi = np.asarray(psi, np.float64)
    b = np.floor((psi - lo) / (hi - lo) * n_bins)
    b = np.where(np.isfinite(psi), b, 0.0)
    b = np.clip(b, 0, n_bins - 1).astype(np.int64)
    counts = np.zeros((psi.shape[0], n_bins), np.int64)
    for r in range(psi.shape[0]):
        np.add.at(counts[r], b[r], 1)
    return counts, np.log1p(counts.astype(np.float64))


def rounded(theta):
    """The parameters the forward pass uses: weights rounded to bfloat16,
    biases as float32 values (packed, float64)."""
    p = unpack(np.asarray(theta, np.float64))
    q = {name: (bf16_round(p[name]) if name in ("W1", "W2", "w3")
                else np.asarray(p[name], np.float32).astype(np.float64)) for name, _ in SIZES}
    return np.concatenate([q[name].ravel() for name, _ in SIZES])


def mlp_forward_raw(params, X):
    """(H1, H2, y) of the packed parameters as given, in FP64."""
    p = unpack(params)
    X = np.asarray(X, np.float64)
    H1 = np.maximum(X @ p["W1"] + p["b1"], 0.0)
    H2 = np.maximum(H1 @ p["W2"] + p["b2"], 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return H1, H2, y


def mlp_forward(theta, X):
    """(H1, H2, y) with bfloat16-rounded weights and FP64 arithmetic."""
    return mlp_forward_raw(rounded(theta), X)


def mlp_backward(theta, X, H1, H2, dy):
    """Packed gradient of a loss with dL/dy = dy with respect to the
    parameters the forward pass used (the rounded ones)."""
    p = unpack(rounded(theta))
    W2, w3 = p["W2"], p["w3"]
    X = np.asarray(X, np.float64)
    dy = np.asarray(dy, np.float64)
    g = {}
    g["w3"] = H2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dZ2 = np.outer(dy, w3) * (H2 > 0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * (H1 > 0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return np.concatenate([g[name].ravel() for name, _ in SIZES])


def bce_with_logits(y, label, pw=1.0):
    """Mean of pw*l*softplus(-y) + (1-l)*softplus(y), and its derivative in y."""
    y = np.asarray(y, np.float64)
    label = np.asarray(label, np.float64)
    sp_pos = np.logaddexp(0.0, y)     # softplus(y)
    sp_neg = np.logaddexp(0.0, -y)    # softplus(-y)
    n = y.shape[0]
    loss = (pw * label * sp_neg + (1.0 - label) * sp_pos).sum() / n
    sig = 1.0 / (1.0 + np.exp(-y))
    dy = (pw * label * (sig - 1.0) + (1.0 - label) * sig) / n
    return loss, dy


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
