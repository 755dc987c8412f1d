"""GPU parity of the training-step services against oracle/train.py:
population-control statistic (float32 sums within 1e-6 relative, counts exact),
plan (actions, offsets and total bit-exact, including exact ties at every
threshold), rewrite (network rows bit for bit, split centres within FP32
rounding, child log-scales bit-exact), the anisotropy regulariser (loss and
gradient) and the fused Adam step (FP32 weights, and BF16 weights with an FP32
master copy); then a few full training steps on a small scene must lower the
loss."""
import math

import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _packed(color="sh", n=3000, seed=3, dynamic=False, bf16=False):
    from paper_2510_08491_gb300.render import pack_scene
    sc = synth.make_scene(n, seed=seed, center_half=2.0, n_sigma=8, omega0=30.0, color=color, dynamic=dynamic,
                          log_scale_mean=-2.5, log_scale_std=0.8)
    if bf16:
        sc = sc.to_bf16()
    return sc, pack_scene(sc)


@pytest.mark.parametrize("color,dynamic", [("sh", False), ("const", True), ("mlp", False)])
def test_statistic_matches_oracle(R, color, dynamic):
    from oracle import train as T
    from paper_2510_08491_gb300.render import unpack_net_grad
    sc, ps = _packed(color, dynamic=dynamic)
    n = sc.n
    rng = np.random.default_rng(11)
    s = torch.zeros(n, dtype=torch.float32, device="cuda")
    c = torch.zeros(n, dtype=torch.int32, device="cuda")
    rs, rc = np.zeros(n), np.zeros(n, np.int64)
    for step in range(3):
        g = rng.normal(size=(n, ps.stride)).astype(np.float32) * np.float32(10.0 ** rng.uniform(-6, 0, size=(n, 1)))
        g[rng.random(n) < 0.2] = 0.0   # primitives that got no gradient this step
        gt = torch.tensor(g, device="cuda")
        R.popctl_accumulate(ps, gt, s, c)
        named = unpack_net_grad(ps, gt, sc)
        rs, rc = T.popctl_accumulate(rs, rc, T.popctl_statistic(named, n))
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), rc)
    assert np.allclose(s.cpu().numpy(), rs, rtol=1e-6, atol=0)


def test_plan_is_bit_exact(R):
    from paper_2510_08491_gb300 import _lib as L
    from oracle import train as T
    sc, ps = _packed("sh", n=20000, seed=5)
    n = sc.n
    rng = np.random.default_rng(12)
    cnt = rng.integers(0, 8, size=n).astype(np.int32)
    s = (rng.exponential(2e-5, size=n) * cnt).astype(np.float32)
    # exact ties: sum == threshold * count in float32
    tie = rng.random(n) < 0.05
    s[tie] = np.float32(1e-5) * cnt[tie].astype(np.float32)
    tie2 = rng.random(n) < 0.05
    s[tie2] = np.float32(1e-6) * cnt[tie2].astype(np.float32)
    cfg = L.PopctlConfig(1e-5, 1e-6, 1e-2, 0.5, 4.0, 0)
    # exact ties on the scale thresholds
    ls = sc.log_scales.copy()
    lg = np.float32(math.log(float(np.float32(1e-2)) * 4.0))
    ls[:50, 0] = lg
    ls[:50, 1:] = lg - 1
    sc.log_scales = ls
    from paper_2510_08491_gb300.render import pack_scene
    ps = pack_scene(sc)
    action, offset, n_out = R.popctl_plan(ps, torch.tensor(s, device="cuda"), torch.tensor(cnt, device="cuda"), cfg)
    ra, ro, rn = T.popctl_plan(sc.log_scales, s, cnt, 1e-5, 1e-6, 1e-2, 0.5, 4.0)
    assert np.array_equal(action.cpu().numpy(), ra)
    assert np.array_equal(offset.cpu().numpy().view(np.uint32).astype(np.int64), ro)
    assert n_out == rn
    assert len(set(ra.tolist())) == 4


@pytest.mark.parametrize("bf16", [False, True])
def test_apply_matches_oracle(R, bf16):
    from oracle import train as T
    sc, ps = _packed("sh", n=5000, seed=6, bf16=bf16)
    n = sc.n
    rng = np.random.default_rng(13)
    action = rng.integers(0, 4, size=n).astype(np.int32)
    offs = np.concatenate([[0], np.cumsum(np.array([0, 1, 2, 2])[action])[:-1]]).astype(np.uint32)
    n_out = int(np.array([0, 1, 2, 2])[action].sum())
    noise = rng.normal(size=(n, 2, 3)).astype(np.float32)
    new = R.popctl_apply(ps, torch.tensor(action, device="cuda"),
                         torch.tensor(offs.view(np.int32), device="cuda"), n_out,
                         torch.tensor(noise, device="cuda"))
    torch.cuda.synchronize()
    fields = {"centers": sc.centers, "log_scales": sc.log_scales, "quats": sc.quats, "rgb": sc.rgb}
    ref, src = T.popctl_apply(fields, action, noise.astype(np.float64))
    g = new.geom.cpu().numpy()
    assert new.n == n_out == len(src)
    # network rows and non-geometric columns copied bit for bit
    assert torch.equal(new.net.cpu(), ps.net.cpu()[torch.tensor(src)])
    assert np.array_equal(g[:, 6:16], ps.geom.cpu().numpy()[src, 6:16])
    assert np.array_equal(g[:, 3:6], ref["log_scales"])
    split = action[src] == T.SPLIT
    assert np.array_equal(g[~split, 0:3], sc.centers[src[~split]])
    err = np.abs(g[split, 0:3] - ref["centers"][split]).max()
    assert err < 2e-6, err


def test_geom_reg_matches_oracle(R):
    from oracle import train as T
    sc, ps = _packed("sh", n=30000, seed=7)
    iso = np.arange(0, 30000, 97)
    ls = sc.log_scales.copy()
    ls[iso] = ls[iso, :1]
    sc.log_scales = ls
    from paper_2510_08491_gb300.render import pack_scene, unpack_geom_grad
    ps = pack_scene(sc)
    base = np.float32(1e-6)
    g = torch.zeros_like(ps.geom)
    g[:, 3:6] = float(base)   # accumulated into
    loss = R.geom_reg(ps, 0.7, g)
    torch.cuda.synchronize()
    rl, rg = T.geom_reg(sc.log_scales, 0.7)
    assert abs(float(loss.item()) - rl) <= 1e-6 * abs(rl)
    gg = unpack_geom_grad(g)["log_scales"] - float(base)
    scale = np.abs(rg).max()
    assert np.abs(gg - rg).max() <= 1e-5 * scale
    assert np.all(gg[iso] == 0.0)


@pytest.mark.parametrize("bf16", [False, True])
def test_adam_matches_oracle(R, bf16):
    from paper_2510_08491_gb300 import _lib as L
    from oracle import train as T
    sc, ps = _packed("sh", n=4000, seed=8, dynamic=True, bf16=bf16)
    n, stride = sc.n, ps.stride
    rng = np.random.default_rng(14)
    lr_geom = [1.6e-4, 5e-3, 1e-3, 2.5e-3]
    lr_net = [1e-3] * 4 + [0.0] * 7 + [2.5e-3, 1e-3, 2.5e-3]
    cfg = L.AdamConfig()
    cfg.lr_geom[:] = lr_geom
    cfg.lr_net[:] = lr_net
    cfg.beta1, cfg.beta2, cfg.eps = 0.9, 0.999, 1e-15
    # the oracle runs on the configuration's float32 values
    f32 = lambda x: float(np.float32(x))
    b1, b2, ep = f32(0.9), f32(0.999), f32(1e-15)
    lr_geom, lr_net = [f32(x) for x in lr_geom], [f32(x) for x in lr_net]
    geom0 = ps.geom.cpu().numpy().astype(np.float64)
    master0 = ps.net.float().cpu().numpy().astype(np.float64)
    master = ps.net.float().clone() if bf16 else None
    mg, vg = torch.zeros_like(ps.geom), torch.zeros_like(ps.geom)
    mn = torch.zeros((n, stride), dtype=torch.float32, device="cuda")
    vn = torch.zeros_like(mn)
    # per-column rates (padding columns follow their field; here all padding gradients are 0)
    col_geom = np.zeros(16)
    col_geom[0:3], col_geom[3:6], col_geom[6:10], col_geom[10:13] = lr_geom
    sizes = [3 * 8, 8, 8, 1, 8, 0, 0, 0, 0, 0, 0, 48, 8, 36]
    col_net = np.zeros(stride)
    valid = np.zeros(stride, bool)
    for k, o in enumerate(ps.offsets):
        if o >= 0:
            col_net[o:o + sizes[k]] = lr_net[k]
            valid[o:o + sizes[k]] = True
    rp, rm, rv = geom0.copy(), np.zeros_like(geom0), np.zeros_like(geom0)
    qp, qm, qv = master0.copy(), np.zeros_like(master0), np.zeros_like(master0)
    for t in (1, 2, 3):
        gg = rng.normal(size=(n, 16)).astype(np.float32) * np.float32(1e-2)
        gn = (rng.normal(size=(n, stride)) * valid).astype(np.float32)
        cfg.step = t
        R.adam_step(ps, torch.tensor(gg, device="cuda"), torch.tensor(gn, device="cuda"), mg, vg, mn, vn, cfg,
                    net_master=master)
        rp2, rm, rv = T.adam(rp, gg, rm, rv, col_geom[None], b1, b2, ep, t)
        rp = np.where(np.arange(16)[None] < 13, rp2, rp)
        qp, qm, qv = T.adam(qp, gn, qm, qv, col_net[None], b1, b2, ep, t)
    torch.cuda.synchronize()
    p = ps.geom.cpu().numpy()
    assert np.abs(p - rp).max() <= 2e-7 * np.abs(rp).max() + 1e-5 * max(lr_geom)
    assert np.array_equal(p[:, 13:], geom0[:, 13:].astype(np.float32))
    assert np.allclose(mg.cpu().numpy()[:, :13], rm[:, :13], rtol=1e-5, atol=1e-9)
    assert np.all(mg.cpu().numpy()[:, 13:] == 0.0)   # unused columns untouched
    w = (master if bf16 else ps.net).float().cpu().numpy()
    assert np.abs(w - qp).max() <= 2e-7 * np.abs(qp).max() + 1e-5 * 2.5e-3
    assert np.allclose(vn.cpu().numpy(), qv, rtol=1e-5, atol=1e-12)
    if bf16:
        assert np.array_equal(ps.net.float().cpu().numpy(), synth.bf16_round(w))


def test_training_steps_lower_the_loss(R):
    """Forward, squared error, backward, regulariser, Adam and the statistic, five
    times on a small scene fitted to a perturbed copy of itself."""
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    sc = synth.make_scene(2000, seed=9, center_half=1.5, n_sigma=8, omega0=30.0, color="sh")
    target = synth.perturb(sc, seed=10, std=0.05)
    cams = synth.ring_cameras(2, 6.0, 96, 96)
    cfg = L.make_config()
    tgt = R.forward(pack_scene(target), cams, cfg).clone()
    ps = pack_scene(sc)
    n, stride = sc.n, ps.stride
    mg, vg = torch.zeros_like(ps.geom), torch.zeros_like(ps.geom)
    mn = torch.zeros((n, stride), dtype=torch.float32, device="cuda")
    vn = torch.zeros_like(mn)
    ssum = torch.zeros(n, dtype=torch.float32, device="cuda")
    scnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    ac = L.AdamConfig()
    ac.lr_geom[:] = [1.6e-4, 5e-3, 1e-3, 0.0]
    ac.lr_net[:] = [1e-3] * 4 + [0.0] * 7 + [2.5e-3, 0.0, 0.0]
    ac.beta1, ac.beta2, ac.eps = 0.9, 0.999, 1e-15
    losses = []
    for t in range(1, 7):
        img = R.forward(ps, cams, cfg)
        loss, dL = R.mse_loss(img, tgt)
        losses.append(float(loss.item()))
        g_geom = torch.zeros_like(ps.geom)
        g_net = torch.zeros((n, stride), dtype=torch.float32, device="cuda")
        R.backward(ps, dL, g_geom, g_net)
        R.geom_reg(ps, 1e-4, g_geom)
        R.popctl_accumulate(ps, g_net, ssum, scnt)
        ac.step = t
        R.adam_step(ps, g_geom, g_net, mg, vg, mn, vn, ac)
    torch.cuda.synchronize()
    assert losses[-1] < 0.9 * losses[0], losses
    assert int((scnt > 0).sum().item()) > 100
