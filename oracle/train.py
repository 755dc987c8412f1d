"""FP64 oracle of the training-step services around the renderer.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy on named
parameter arrays (the synth.Scene fields), no packed layouts:

  * popctl_statistic / popctl_accumulate -- Sec. 3.3, Population Control: the
    densification criterion is the gradient magnitude of each primitive's network
    weights (here the density network: W1, b1, w2, b2 and, for a time-conditioned
    scene, W_t), accumulated over the steps in which the primitive got gradient.
  * popctl_plan -- the clone / split / prune decision with the thresholds of App.
    hyperparameters (gradient threshold, pruning threshold, growing scale threshold,
    pruning scale threshold), in the rule order the library documents.  The
    comparisons that decide an integer are taken in float32, as the library takes
    them: both sides must make the same decision on the same inputs.
  * popctl_apply -- the new primitive set: survivors in order, clones duplicated,
    split parents replaced by two children placed at c + R(q) diag(s) eps_j with
    scales divided by 1.6 (the split of 3D Gaussian splatting, which the paper says
    it follows).
  * geom_reg -- Sec. 3.3 Training / Sec. 5.3: the standard deviation of the
    components of each scale vector s = exp(log s), averaged over primitives, and
    its gradient with respect to the log-scales.
  * adam -- Kingma and Ba, "Adam", Algorithm 1 (bias-corrected first and second
    moment estimates), the optimiser the paper trains with (App. hyperparameters).
"""
from __future__ import annotations

import math
from typing import Dict

import numpy as np

PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3
DENSITY_FIELDS = ("W1", "b1", "w2", "b2", "wt")


def popctl_statistic(grads: Dict[str, np.ndarray], n: int) -> np.ndarray:
    """m_i = || gradient of primitive i's density-network weights ||_2 (float64)."""
    sq = np.zeros(n, np.float64)
    for f in DENSITY_FIELDS:
        if f in grads and grads[f] is not None:
            g = np.asarray(grads[f], np.float64).reshape(n, -1)
            sq += (g * g).sum(axis=1)
    return np.sqrt(sq)


def popctl_accumulate(stat_sum: np.ndarray, stat_count: np.ndarray, m: np.ndarray):
    """Where m_i > 0: sum_i += m_i, count_i += 1 (returns new arrays)."""
    on = m > 0
    s = np.asarray(stat_sum, np.float64) + np.where(on, m, 0.0)
    c = np.asarray(stat_count, np.int64) + on.astype(np.int64)
    return s, c


def popctl_plan(log_scales: np.ndarray, stat_sum: np.ndarray, stat_count: np.ndarray, grad_threshold: float,
                prune_threshold: float, grow_scale: float, prune_scale: float, extent: float):
    """Action per primitive and the first output row of each (exclusive scan of
    0 / 1 / 2 / 2 outputs for prune / keep / clone / split) and the total.

    Rules, first that applies, with l = max(log s):
      l > ln(prune_scale * extent)                      -> prune (too large)
      count > 0 and sum >= grad_threshold * count       -> clone if l <= ln(grow_scale * extent) else split
      count == 0 or sum < prune_threshold * count       -> prune (low gradient)
      otherwise                                         -> keep
    All comparisons in float32; the products grad_threshold * count in float32; the
    two logarithms in double, rounded to float32."""
    f32 = np.float32
    l = np.asarray(log_scales, f32).max(axis=1)
    s = np.asarray(stat_sum, f32)
    c = np.asarray(stat_count, np.int64)
    cf = c.astype(f32)
    log_prune = f32(math.log(float(f32(prune_scale)) * float(f32(extent))))
    log_grow = f32(math.log(float(f32(grow_scale)) * float(f32(extent))))
    dens = (c > 0) & (s >= f32(grad_threshold) * cf)
    low = (c == 0) | (s < f32(prune_threshold) * cf)
    action = np.full(len(l), KEEP, np.int32)
    action[low] = PRUNE
    action[dens] = np.where(l[dens] <= log_grow, CLONE, SPLIT)
    action[l > log_prune] = PRUNE
    outs = np.array([0, 1, 2, 2], np.int64)[action]
    offset = np.concatenate([[0], np.cumsum(outs)[:-1]]) if len(outs) else np.zeros(0, np.int64)
    return action, offset.astype(np.int64), int(outs.sum())


def rotation(q: np.ndarray) -> np.ndarray:
    """R(q) for q = (w, x, y, z), normalised first (float64, [n, 3, 3])."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=-1)
    return R.reshape(q.shape[:-1] + (3, 3))


def popctl_apply(fields: Dict[str, np.ndarray], action: np.ndarray, noise: np.ndarray):
    """New parameter arrays.  Survivors keep their order; a clone is two copies; a
    split parent becomes two children j = 0, 1 with centre c + R(q) diag(s) eps_j
    (s = exp(log s), float64) and log-scales log s - fl32(ln 1.6) (float32
    subtraction); every other field is copied."""
    reps = np.array([0, 1, 2, 2])[np.asarray(action)]
    src = np.repeat(np.arange(len(action)), reps)
    j = np.arange(len(src)) - np.repeat(np.cumsum(reps) - reps, reps)
    out = {k: np.asarray(v)[src].copy() for k, v in fields.items()}
    split = np.asarray(action)[src] == SPLIT
    if split.any():
        p = src[split]
        s = np.exp(np.asarray(fields["log_scales"], np.float64)[p])
        eps = np.asarray(noise, np.float64)[p, j[split]]
        R = rotation(np.asarray(fields["quats"], np.float64)[p])
        c = np.asarray(fields["centers"], np.float64)[p] + np.einsum("qab,qb->qa", R, s * eps)
        out["centers"] = out["centers"].astype(np.float64)
        out["centers"][split] = c
        ls = np.asarray(fields["log_scales"], np.float32)[p]
        out["log_scales"] = out["log_scales"].astype(np.float32)
        out["log_scales"][split] = ls - np.float32(math.log(1.6))
    return out, src


def geom_reg(log_scales: np.ndarray, weight: float):
    """L = weight * mean_i std(s_i), std over the three components (population form),
    and dL/dlog s (0 for isotropic primitives, where std is not differentiable)."""
    s = np.exp(np.asarray(log_scales, np.float64))
    n = len(s)
    if n == 0:
        return 0.0, np.zeros((0, 3))
    mu = s.mean(axis=1, keepdims=True)
    sd = np.sqrt(((s - mu) ** 2).mean(axis=1))
    # an isotropic primitive has std exactly 0 (the rounded mean of three equal
    # values can miss them by an ulp, which would leave a spurious tiny std)
    sd[(s[:, 0] == s[:, 1]) & (s[:, 1] == s[:, 2])] = 0.0
    loss = weight * sd.mean()
    safe = np.where(sd > 0, sd, 1.0)
    g = np.where(sd[:, None] > 0, (weight / n) * s * (s - mu) / (3.0 * safe[:, None]), 0.0)
    return float(loss), g


def adam(p, g, m, v, lr, beta1: float, beta2: float, eps: float, t: int):
    """One step of Adam (Algorithm 1): returns (p, m, v), all float64."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - np.asarray(lr, np.float64) * mhat / (np.sqrt(vhat) + eps), m, v
