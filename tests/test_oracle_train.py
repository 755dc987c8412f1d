"""Pins for the training-step oracle (oracle/train.py): population control
(Sec. 3.3), the anisotropy regulariser (Sec. 3.3 Training, Sec. 5.3) and Adam.

Each check compares the oracle with something other than itself: numpy's norm
and std, central finite differences, torch.optim.Adam, scipy's rotations, an
element-by-element if/elif restatement of the decision rules on hand-built
cases (including exact ties at every threshold), and closed-form cases.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import train as T


def test_statistic_is_the_density_gradient_norm():
    rng = np.random.default_rng(0)
    n, ns = 50, 8
    g = {"W1": rng.normal(size=(n, ns, 3)), "b1": rng.normal(size=(n, ns)), "w2": rng.normal(size=(n, ns)),
         "b2": rng.normal(size=n), "sh": rng.normal(size=(n, 16, 3))}
    for k in ("W1", "b1", "w2", "b2"):
        g[k][7] = 0.0
    m = T.popctl_statistic(g, n)
    flat = np.concatenate([g["W1"].reshape(n, -1), g["b1"], g["w2"], g["b2"][:, None]], axis=1)
    assert np.allclose(m, np.linalg.norm(flat, axis=1), rtol=1e-14)   # colour coefficients excluded
    s, c = T.popctl_accumulate(np.zeros(n), np.zeros(n, np.int64), m)
    s, c = T.popctl_accumulate(s, c, m)
    assert c[7] == 0 and s[7] == 0.0 and np.all(c[np.arange(n) != 7] == 2)
    assert np.allclose(s, 2 * m)
    g["wt"] = rng.normal(size=(n, ns))
    m2 = T.popctl_statistic(g, n)
    assert np.allclose(m2 ** 2, m ** 2 + (g["wt"] ** 2).sum(axis=1))


def _rules_loop(l, s, c, gt, pt, gs, ps, ext):
    """The decision written out element by element in the documented rule order."""
    f32 = np.float32
    lp = f32(math.log(float(f32(ps)) * float(f32(ext))))
    lg = f32(math.log(float(f32(gs)) * float(f32(ext))))
    out = []
    for li, si, ci in zip(l, s, c):
        if li > lp:
            out.append(T.PRUNE)
        elif ci > 0 and si >= f32(gt) * f32(ci):
            out.append(T.CLONE if li <= lg else T.SPLIT)
        elif ci == 0 or si < f32(pt) * f32(ci):
            out.append(T.PRUNE)
        else:
            out.append(T.KEEP)
    return np.array(out, np.int32)


def test_plan_rules_and_ties():
    f32 = np.float32
    gt, pt, gs, ps, ext = 0.25, 0.0625, 0.01, 0.5, 3.0
    lg = f32(math.log(gs * float(f32(ext))))
    lp = f32(math.log(ps * float(f32(ext))))
    small, mid = f32(lg - 1.0), f32((lg + lp) / 2)
    # (max log-scale, sum, count) -> expected action
    cases = [
        (small, 1.0, 4, T.CLONE),                      # sum == 0.25 * 4 exactly: densify (>=)
        (np.nextafter(lg, f32(-1e9)), 2.0, 4, T.CLONE),
        (lg, 2.0, 4, T.CLONE),                         # l == ln(grow * extent): clone (<=)
        (np.nextafter(lg, f32(1e9)), 2.0, 4, T.SPLIT),
        (mid, 5.0, 4, T.SPLIT),
        (lp, 5.0, 4, T.SPLIT),                         # l == ln(prune * extent): not too large
        (np.nextafter(lp, f32(1e9)), 5.0, 4, T.PRUNE),  # too large wins over densify
        (mid, 0.0, 0, T.PRUNE),                        # never saw gradient
        (mid, 0.25, 4, T.KEEP),                        # sum == 0.0625 * 4: not below
        (mid, float(np.nextafter(f32(0.25), f32(0))), 4, T.PRUNE),
        (mid, 0.5, 4, T.KEEP),
        (mid, float(np.nextafter(f32(1.0), f32(0))), 4, T.KEEP),
    ]
    ls = np.zeros((len(cases), 3), np.float32)
    ls[:, 1] = [c[0] for c in cases]
    ls[:, 0] = ls[:, 1] - 1.0
    ls[:, 2] = ls[:, 1] - 2.0
    s = np.array([c[1] for c in cases], np.float32)
    cnt = np.array([c[2] for c in cases], np.int32)
    act, off, total = T.popctl_plan(ls, s, cnt, gt, pt, gs, ps, ext)
    assert list(act) == [c[3] for c in cases]
    assert total == sum({T.PRUNE: 0, T.KEEP: 1, T.CLONE: 2, T.SPLIT: 2}[a] for a in act)
    assert list(off) == list(np.concatenate([[0], np.cumsum([[0, 1, 2, 2][a] for a in act])[:-1]]))


def test_plan_matches_loop_on_random_inputs():
    rng = np.random.default_rng(3)
    n = 4000
    ls = rng.normal(-3.0, 1.5, size=(n, 3)).astype(np.float32)
    cnt = rng.integers(0, 6, size=n).astype(np.int32)
    s = (rng.exponential(3e-5, size=n) * cnt).astype(np.float32)
    args = (1e-5, 1e-6, 1e-2, 0.5, 2.0)
    act, off, total = T.popctl_plan(ls, s, cnt, *args)
    ref = _rules_loop(ls.max(axis=1), s, cnt, *args)
    assert np.array_equal(act, ref)
    assert len(set(act.tolist())) == 4
    assert off[-1] + [0, 1, 2, 2][act[-1]] == total


def test_apply_children_and_copies():
    rng = np.random.default_rng(5)
    n = 40
    f = {"centers": rng.normal(size=(n, 3)).astype(np.float32),
         "log_scales": rng.normal(-2, 0.5, size=(n, 3)).astype(np.float32),
         "quats": rng.normal(size=(n, 4)).astype(np.float32),
         "W1": rng.normal(size=(n, 8, 3)).astype(np.float32), "b2": rng.normal(size=n).astype(np.float32)}
    action = rng.integers(0, 4, size=n).astype(np.int32)
    noise = rng.normal(size=(n, 2, 3))
    out, src = T.popctl_apply(f, action, noise)
    assert len(src) == sum([0, 1, 2, 2][a] for a in action)
    assert np.all(np.diff(src) >= 0)                         # survivors keep their order
    assert set(src.tolist()) == set(np.nonzero(action != T.PRUNE)[0].tolist())
    for k in ("W1", "b2", "quats"):
        assert np.array_equal(out[k], f[k][src])
    seen = {}
    for r, p in enumerate(src):
        j = seen.get(p, 0)
        seen[p] = j + 1
        if action[p] == T.SPLIT:
            # the child's offset in the parent's frame (scipy rotation) is diag(s) eps_j
            q = f["quats"][p].astype(np.float64)
            Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
            local = Rm.T @ (out["centers"][r] - f["centers"][p].astype(np.float64))
            assert np.allclose(local, np.exp(f["log_scales"][p].astype(np.float64)) * noise[p, j], atol=1e-12)
            assert np.allclose(np.exp(out["log_scales"][r].astype(np.float64)),
                               np.exp(f["log_scales"][p].astype(np.float64)) / 1.6, rtol=2e-7)
        else:
            assert np.array_equal(out["centers"][r], f["centers"][p])
            assert np.array_equal(out["log_scales"][r], f["log_scales"][p])
    # zero noise: both children sit at the parent's centre
    out0, src0 = T.popctl_apply(f, np.full(n, T.SPLIT, np.int32), np.zeros((n, 2, 3)))
    assert np.allclose(out0["centers"], f["centers"][src0], atol=0)


def test_geom_reg_closed_forms_and_gradient():
    rng = np.random.default_rng(7)
    ls = rng.normal(-2, 0.6, size=(30, 3))
    w = 0.3
    loss, g = T.geom_reg(ls, w)
    assert math.isclose(loss, w * np.std(np.exp(ls), axis=1).mean(), rel_tol=1e-13)
    # central differences
    h = 1e-6
    for i, a in [(0, 0), (3, 2), (17, 1), (29, 0)]:
        p, m = ls.copy(), ls.copy()
        p[i, a] += h
        m[i, a] -= h
        fd = (T.geom_reg(p, w)[0] - T.geom_reg(m, w)[0]) / (2 * h)
        assert abs(fd - g[i, a]) < 1e-8 * max(1.0, abs(g[i, a]))
    # isotropic primitives: no penalty and zero gradient (many rows, so that some
    # have a mean that float64 rounds away from the common value)
    iso = np.repeat(rng.normal(-2, 0.8, size=(1000, 1)).astype(np.float32), 3, axis=1)
    s_iso = np.exp(iso.astype(np.float64))
    assert np.any(s_iso.mean(axis=1) != s_iso[:, 0])
    l0, g0 = T.geom_reg(iso, w)
    assert l0 == 0.0 and np.all(g0 == 0.0)
    # scaling every primitive by k scales the penalty by k
    l2, _ = T.geom_reg(ls + math.log(2.5), w)
    assert math.isclose(l2, 2.5 * loss, rel_tol=1e-12)
    # two equal axes and one twice as long: std = (sqrt(2)/3) a
    l3, _ = T.geom_reg(np.log(np.array([[0.1, 0.1, 0.2]])), 1.0)
    assert math.isclose(l3, math.sqrt(2.0) / 3.0 * 0.1, rel_tol=1e-12)


def test_adam_matches_torch():
    rng = np.random.default_rng(9)
    p0 = rng.normal(size=(6, 7))
    lr = np.array([1e-3, 1e-3, 5e-3, 5e-3, 1.6e-4, 2.5e-3, 0.0])
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    groups = [{"params": [], "lr": float(x)} for x in lr]
    cols = [torch.tensor(p0[:, j:j + 1], dtype=torch.float64, requires_grad=True) for j in range(7)]
    for j, grp in enumerate(groups):
        grp["params"] = [cols[j]]
    opt = torch.optim.Adam(groups, betas=(0.9, 0.999), eps=1e-15)
    mine, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 5):
        g = rng.normal(size=p0.shape)
        for j in range(7):
            cols[j].grad = torch.tensor(g[:, j:j + 1], dtype=torch.float64)
        opt.step()
        mine, m, v = T.adam(mine, g, m, v, lr[None, :], 0.9, 0.999, 1e-15, t)
    ref = np.concatenate([c.detach().numpy() for c in cols], axis=1)
    assert np.abs(mine - ref).max() < 1e-14
    assert np.array_equal(mine[:, 6], p0[:, 6])   # zero rate: untouched
    del p


def _golden(name):
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("="))
            vals[k] = float(v)
    return vals


def test_bench_uses_the_papers_hyperparameters():
    """The training-step benchmark's Adam rates and population-control thresholds
    are the paper's (App. hyperparameters), field by field; the dynamic series has
    the printed number of terms."""
    import bench
    g = _golden("paper_hyperparameters.txt")
    assert bench.PAPER_LR_GEOM[:3] == [g["lr_means"], g["lr_scales"], g["lr_quats"]]
    net = bench.PAPER_LR_NET
    assert net[0:4] == [g["lr_mlp"]] * 4           # W1, b1, w2, b2
    assert net[4:11] == [g["lr_mlp"]] * 7          # colour MLP fields
    assert net[11] == g["lr_sh"] and net[13] == g["lr_sh"]  # sh, degree-0 series
    assert bench.PAPER_POPCTL_SYNTHETIC == (g["densify_synthetic"], g["prune_synthetic"], g["grow_scale"],
                                           g["prune_scale"])
    from oracle import grad as Gd
    # the degree-0 series: xi^j (j = 1..n) and cos(j xi), sin(j xi) (j = 1..l)
    assert len(Gd._time_series(0.3)) == g["series_poly_terms"] + 2 * g["series_fourier_terms"]
