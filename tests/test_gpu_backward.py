"""GPU parity of the backward pass through the C ABI against the FP64 gradient oracle.

Bar: per parameter group, |g - g*| <= 1e-3 (|g*| + rms(g*)) elementwise and
||g - g*|| / ||g*|| <= 1e-3, for centres, log-scales, quaternions, constant
colours and every density / colour-MLP weight.  dL/dC is a seeded random image.
Pixels whose termination step is a near-tie (|T - T_min| < 1% T_min), where FP32
may decide differently from FP64, get dL = 0.  No silhouette band is needed: the
kernels evaluate the ray geometry relative to the ray through each primitive's
centre (FP32 h^2 error ~1e-7) and re-evaluate pairs with |h^2| < 1e-2 in
float-float arithmetic, so the 1 / sqrt(h^2) growth of the derivative near a
silhouette is followed.  The _dl helper keeps a sil_eps option for diagnostics.

The colour MLP's hidden layer runs on the tensor cores with split-bf16 operands
(about 1e-5 relative per product), so a ReLU pre-activation within ~1e-5 of zero
may be decided differently from FP64.  The gradient is discontinuous there (the
ReLU kink), so, like the termination near-ties, pixels with a composited pair
whose smallest |pre-activation| is below RELU_EPS = 1e-4 get dL = 0 (about 1% of
the pixels of these scenes).
"""
import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth
from gpu_util import grad_rel_errors

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
SIL_EPS = 0.0
RELU_EPS = 1e-4


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _gpu_grads(R, scene, cams, dL, form=0, t_min=1e-4, bg=(0.0, 0.0, 0.0)):
    return _gpu_grads_cfg(R, scene, cams, dL, form=form, t_min=t_min, bg=bg)


def _gpu_grads_cfg(R, scene, cams, dL, **cfg_kw):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene, unpack_geom_grad, unpack_net_grad
    ps = pack_scene(scene)
    cfg = L.make_config(**cfg_kw)
    R.forward(ps, cams, cfg)
    g_geom = torch.zeros_like(ps.geom)
    g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device=ps.net.device)
    R.backward(ps, torch.tensor(dL, dtype=torch.float32, device="cuda"), g_geom, g_net)
    torch.cuda.synchronize()
    g = unpack_geom_grad(g_geom)
    g.update(unpack_net_grad(ps, g_net, scene))
    return g


def _oracle_grads(O, scene, cams, dL_views, t_min=1e-4, bg=(0.0, 0.0, 0.0), ts=16):
    from oracle import grad as G
    tl = O.tile_keys(scene, cams, ts)
    lp = (tl.vals.astype(np.int64) % scene.n).astype(np.int32)
    total = None
    for v, cam in enumerate(cams):
        pix = np.arange(cam.n_pixels, dtype=np.int32)
        gt = tl.view_tile_off[v] + O.pixel_tile(cam, ts, pix)
        _, g = G.grads(scene, cam, pix, gt, tl.tile_off, lp, dL_views[v], t_min, bg)
        total = g if total is None else {k: total[k] + g[k] for k in g}
    return total


def _dl(O, scene, cams, seed, t_min=1e-4, bg=(0.0, 0.0, 0.0), sil_eps=SIL_EPS, relu_eps=RELU_EPS):
    """Seeded dL/dC, zero on near-tie termination pixels, on pixels with a pair at
    a colour-MLP ReLU kink (|pre-activation| < relu_eps) and, for diagnostics, on
    near-silhouette pixels (|h^2| < sil_eps)."""
    from oracle import grad as G
    rng = np.random.default_rng(seed)
    imgs, tl, outs = O.render_image(scene, cams, 16, t_min, bg)
    lp = (tl.vals.astype(np.int64) % scene.n).astype(np.int32)
    per_view = []
    for v, (cam, o) in enumerate(zip(cams, outs)):
        d = rng.normal(size=(cam.n_pixels, 3))
        d[o.flags != 0] = 0.0
        if sil_eps > 0 or (relu_eps > 0 and scene.color in ("mlp", "sh")):
            pix = np.arange(cam.n_pixels, dtype=np.int32)
            gt = tl.view_tile_off[v] + O.pixel_tile(cam, 16, pix)
            lens = tl.tile_off[gt + 1] - tl.tile_off[gt]
            owner = np.repeat(np.arange(cam.n_pixels), lens)
            _, h2, ah, amin = G.pair_diagnostics(scene, cam, pix, gt, tl.tile_off, lp)
            near = np.zeros(cam.n_pixels, bool)
            near[owner[np.abs(h2) < sil_eps]] = True
            if scene.color in ("mlp", "sh"):
                near[owner[(ah > 0) & (amin < relu_eps)]] = True
            d[near] = 0.0
        per_view.append(d)
    return per_view


def test_report_silhouette_band(R, oracle_lib):
    """Diagnostic (no assertion): gradient error versus the silhouette band on the dense scene."""
    O = oracle_lib
    sc = synth.make_scene(1200, seed=3, center_half=1.5, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 72, 56)]
    for eps in (0.0, 1e-4, 1e-3, 1e-2, 3e-2):
        dLv = _dl(O, sc, cams, 3, sil_eps=eps)
        g = _gpu_grads(R, sc, cams, np.concatenate(dLv))
        gref = _oracle_grads(O, sc, cams, dLv)
        errs = grad_rel_errors(g, {k: gref[k] for k in ("centers", "log_scales", "quats", "W1", "Wc2")})
        print("sil_eps", eps, {k: (f"{a:.1e}", f"{b:.1e}") for k, (a, b) in errs.items()})


def _check(g, gref, fields):
    errs = grad_rel_errors(g, {k: gref[k] for k in fields})
    print({k: (f"{a:.1e}", f"{b:.1e}") for k, (a, b) in errs.items()})
    bad = {k: v for k, v in errs.items() if v[0] > GRAD_TOL or v[1] > GRAD_TOL}
    assert not bad, f"gradient mismatch: {bad}"
    return errs


def test_const_colour_tiny(R, oracle_lib):
    O = oracle_lib
    wl = synth.workload("tiny64_128px")
    dLv = _dl(O, wl.scene, wl.cameras, 1)
    g = _gpu_grads(R, wl.scene, wl.cameras, np.concatenate(dLv))
    gref = _oracle_grads(O, wl.scene, wl.cameras, dLv)
    _check(g, gref, ["centers", "log_scales", "quats", "rgb", "W1", "b1", "w2", "b2"])


def test_mlp_fd_subset_scene(R, oracle_lib):
    """2,000 primitives with the differentiation workload's distributions, 64 x 64, ring camera k=0."""
    O = oracle_lib
    sc = synth.make_scene(2000, seed=0, center_half=3.0, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
    cams = synth.ring_cameras(1, 8.0, 64, 64)
    dLv = _dl(O, sc, cams, 2)
    g = _gpu_grads(R, sc, cams, np.concatenate(dLv))
    gref = _oracle_grads(O, sc, cams, dLv)
    _check(g, gref, sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"])


def test_mlp_denser_multiview(R, oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(1200, seed=3, center_half=1.5, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 72, 56),
            synth.look_at_camera((6.0, 0.0, 0.0), (0, 0, 0), 50, 61)]
    dLv = _dl(O, sc, cams, 3, bg=(0.2, 0.1, 0.3))
    g = _gpu_grads(R, sc, cams, np.concatenate(dLv), bg=(0.2, 0.1, 0.3))
    gref = _oracle_grads(O, sc, cams, dLv, bg=(0.2, 0.1, 0.3))
    _check(g, gref, sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"])


def test_mlp64_ns32_bf16(R, oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(800, seed=8, center_half=1.5, n_sigma=32, omega0=5.0, color="mlp", n_c=64).to_bf16()
    cams = [synth.look_at_camera((0.0, 0.0, 6.0), (0, 0, 0), 64, 48)]
    dLv = _dl(O, sc, cams, 4)
    g = _gpu_grads(R, sc, cams, np.concatenate(dLv))
    gref = _oracle_grads(O, sc, cams, dLv)
    _check(g, gref, sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"])


@pytest.mark.parametrize("bwd_chunk", [1, 3, 0])
def test_mlp64_backward_chunk_is_set_apart_from_the_forwards(R, oracle_lib, bwd_chunk):
    """The backward's chunk is its own setting (0: the largest that fits, 4 entries
    at N_c = 64 with the tensor-memory dL/dWc2), not bounded by the forward's: with
    the forward at chunk 2, backward chunks of 1, 3 and the default all match the
    oracle.  A negative chunk is refused."""
    from paper_2510_08491_gb300 import _lib as L
    O = oracle_lib
    sc = synth.make_scene(900, seed=18, center_half=1.5, n_sigma=32, omega0=5.0, color="mlp", n_c=64).to_bf16()
    cams = [synth.look_at_camera((0.0, 0.3, 6.0), (0, 0, 0), 72, 40),
            synth.look_at_camera((4.0, 1.0, 4.0), (0, 0, 0), 40, 56)]
    dLv = _dl(O, sc, cams, 6)
    g = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv), chunk=2, bwd_chunk=bwd_chunk)
    _check(g, _oracle_grads(O, sc, cams, dLv),
           sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"])
    if bwd_chunk == 0:
        from paper_2510_08491_gb300.render import pack_scene
        with pytest.raises(L.SnpError) as ei:
            R.forward(pack_scene(sc), cams, L.make_config(bwd_chunk=-1))
        assert ei.value.status == L.SNP_ERR_INVALID_ARG


@pytest.mark.parametrize("replay", [False, True])
def test_mlp_colour_store_and_replay(R, oracle_lib, replay):
    """The backward with the forward's colour store (default) and with the colours
    recomputed (SNP_FLAG_REPLAY_COLOR) both match the oracle, and each other."""
    O = oracle_lib
    sc = synth.make_scene(1500, seed=12, center_half=1.5, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 80, 64),
            synth.look_at_camera((5.0, 1.0, 3.0), (0, 0, 0), 48, 72)]
    dLv = _dl(O, sc, cams, 5)
    fields = sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"]
    g = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv), replay_color=replay)
    _check(g, _oracle_grads(O, sc, cams, dLv), fields)
    g_other = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv), replay_color=not replay)
    for k in fields:
        scale = np.abs(g[k]).max() + 1e-30
        assert np.abs(g[k] - g_other[k]).max() <= 1e-5 * scale, k


def test_mlp_colour_store_partly_full(R, oracle_lib, monkeypatch):
    """A colour store too small for the forward (host-side test hook): the chunks
    whose pairs did not fit are recomputed by the backward; the gradients still
    match the oracle and the fully recomputed backward."""
    O = oracle_lib
    sc = synth.make_scene(1500, seed=14, center_half=1.5, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 80, 64)]
    dLv = _dl(O, sc, cams, 9)
    fields = sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"]
    from paper_2510_08491_gb300.render import pack_scene
    g_replay = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv), replay_color=True)
    R.forward(pack_scene(sc), cams)
    total = R.stats().n_composited
    monkeypatch.setenv("SNP_TEST_COLSTORE_PAIRS", str(total // 3))  # about a third fits
    g = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv))
    _check(g, _oracle_grads(O, sc, cams, dLv), fields)
    for k in fields:
        scale = np.abs(g[k]).max() + 1e-30
        assert np.abs(g[k] - g_replay[k]).max() <= 1e-5 * scale, k


def test_bounded_wait_timeout_is_reported_and_the_context_recovers(R, monkeypatch):
    """The backward at N_c = 64 (tensor-memory accumulation) bounds every wait.  A
    host-side hook (SNP_TEST_STUCK_WAIT) makes one of them wait on a barrier phase
    that nothing completes: the wait gives up, the backward still finishes with the
    same gradients, snp_get_stats reports SNP_ERR_TIMEOUT, and the next forward
    clears the status."""
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    sc = synth.make_scene(800, seed=8, center_half=1.5, n_sigma=32, omega0=5.0, color="mlp", n_c=64).to_bf16()
    cams = [synth.look_at_camera((0.0, 0.0, 6.0), (0, 0, 0), 64, 48)]
    ps = pack_scene(sc)
    dL = torch.randn((cams[0].n_pixels, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(3))

    def run():
        R.forward(ps, cams, L.make_config())
        gg = torch.zeros_like(ps.geom)
        gn = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
        R.backward(ps, dL, gg, gn)
        torch.cuda.synchronize()
        return gg, gn

    ref = run()
    R.stats()
    monkeypatch.setenv("SNP_TEST_STUCK_WAIT", "1")
    got = run()
    with pytest.raises(L.SnpError) as ei:
        R.stats()
    assert ei.value.status == L.SNP_ERR_TIMEOUT
    for a, b in zip(got, ref):
        assert (a - b).abs().max().item() <= 1e-5 * (b.abs().max().item() + 1e-12)
    monkeypatch.delenv("SNP_TEST_STUCK_WAIT")
    again = run()
    R.stats()  # cleared by the forward, and no wait gave up
    for a, b in zip(again, ref):
        assert (a - b).abs().max().item() <= 1e-5 * (b.abs().max().item() + 1e-12)
