"""Parity at the full sizes of the benchmark workloads, in the configuration the
benchmark times (16-pixel tiles, the library's default chunks, colour store on).

* diff300k_720p (300k primitives, colour MLP N_c = 32, 1280 x 720): the backward of
  the full scene with dL/dC set only on a few sampled tiles must equal the FP64
  gradient oracle on the primitives those tiles list (and be exactly zero for every
  other primitive); the forward's keys are bit-exact and the sampled tiles match;
  with dL/dC everywhere, the gradients with the colour store and with the colours
  recomputed agree.
* batch500k_16view (500k primitives, N_sigma = 32, N_c = 64, BF16 weights, 16
  views of uneven size): all 40 M keys bit-exact, sampled tiles of every view
  against the oracle, and colour store vs recomputation at full size.

The oracle runs on the subset of primitives the sampled tiles list (their network
weights in float64 for the whole scene would not fit in host memory)."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth
from gpu_util import assert_image_close, sample_tiles, tile_subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _geometry_only(sc):
    """The scene without its colour network (enough for the key specification)."""
    none = {f: None for f in ("feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3", "sh", "wt", "sh_t")}
    return dataclasses.replace(sc, color="const", n_c=0, dynamic=False, **none)


def _forward_and_keys(R, O, wl):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    ps = pack_scene(wl.scene)
    cfg = L.make_config(tile_size=16, t_min=wl.t_min)
    img = R.forward(ps, wl.cameras, cfg).cpu().numpy()
    keys, vals = R.debug_keys()
    tl = O.tile_keys(_geometry_only(wl.scene), wl.cameras, 16)
    assert np.array_equal(keys, tl.keys)
    assert np.array_equal(vals, tl.vals)
    return ps, cfg, img, tl


def _check_tiles(O, wl, img, tl, picks):
    sub, prims, per_view = tile_subset(O, wl.scene, tl, picks)
    pix_off = np.concatenate([[0], np.cumsum([c.n_pixels for c in wl.cameras])])
    for v, (pix, owner, off, lst) in per_view.items():
        out = O.render_pixels(sub, wl.cameras[v], pix, owner, off, lst, t_min=wl.t_min)
        assert_image_close(img[pix_off[v] + pix], out.rgb, out.flags)
    return sub, prims, per_view


def _store_vs_replay(R, ps, cams, cfg, dL):
    """Full-size gradients with the colour store and with the colours recomputed."""
    from paper_2510_08491_gb300 import _lib as L
    out = []
    for replay in (False, True):
        c = L.make_config(tile_size=int(cfg.tile_size), t_min=float(cfg.t_min), replay_color=replay)
        R.forward(ps, cams, c)
        g_geom = torch.zeros_like(ps.geom)
        g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
        R.backward(ps, dL, g_geom, g_net)
        out.append((g_geom, g_net))
    torch.cuda.synchronize()
    for a, b in zip(out[0], out[1]):
        scale = float(a.abs().max())
        assert float((a - b).abs().max()) <= 1e-5 * scale


def test_full_size_diff300k_backward_on_sampled_tiles(R, oracle_lib):
    from oracle import grad as G
    from paper_2510_08491_gb300.render import unpack_geom_grad, unpack_net_grad
    from test_gpu_backward import GRAD_TOL, RELU_EPS
    from gpu_util import grad_rel_errors
    O = oracle_lib
    wl = synth.workload("diff300k_720p")
    ps, cfg, img, tl = _forward_and_keys(R, O, wl)
    picks = sample_tiles(wl.cameras, tl, 16, 4, seed=21)
    sub, prims, per_view = _check_tiles(O, wl, img, tl, picks)
    cam = wl.cameras[0]
    pix, owner, off, lst = per_view[0]
    # dL/dC on the sampled tiles only, zero on termination near-ties and colour-MLP kinks
    rng = np.random.default_rng(22)
    d = rng.normal(size=(len(pix), 3))
    out = O.render_pixels(sub, cam, pix, owner, off, lst, t_min=wl.t_min)
    d[out.flags != 0] = 0.0
    _, h2, ah, amin = G.pair_diagnostics(sub, cam, pix, owner, off, lst)
    lens = off[owner + 1] - off[owner]
    pair_pix = np.repeat(np.arange(len(pix)), lens)
    d[np.unique(pair_pix[(ah > 0) & (amin < RELU_EPS)])] = 0.0
    dL = np.zeros((cam.n_pixels, 3), np.float32)
    dL[pix] = d
    _, gref = G.grads(sub, cam, pix, owner, off, lst, d, t_min=wl.t_min)
    R.forward(ps, wl.cameras, cfg)
    g_geom = torch.zeros_like(ps.geom)
    g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
    R.backward(ps, torch.tensor(dL, device="cuda"), g_geom, g_net)
    torch.cuda.synchronize()
    g = unpack_geom_grad(g_geom)
    g.update(unpack_net_grad(ps, g_net, wl.scene))
    fields = ["centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3",
              "bc3"]
    others = np.ones(wl.scene.n, bool)
    others[prims] = False
    for f in fields:
        assert not np.any(g[f][others]), f   # no other primitive receives gradient
    errs = grad_rel_errors({f: g[f][prims] for f in fields}, {f: gref[f] for f in fields})
    bad = {k: v for k, v in errs.items() if v[0] > GRAD_TOL or v[1] > GRAD_TOL}
    assert not bad, bad
    # the colour store and the recomputation agree at full size
    dl_all = torch.randn((cam.n_pixels, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    _store_vs_replay(R, ps, wl.cameras, cfg, dl_all * 1e-3)


def test_full_size_batch500k_keys_tiles_and_store(R, oracle_lib):
    O = oracle_lib
    wl = synth.workload("batch500k_16view")
    ps, cfg, img, tl = _forward_and_keys(R, O, wl)
    picks = sample_tiles(wl.cameras, tl, 16, 1, seed=31)
    _check_tiles(O, wl, img, tl, picks)
    P = sum(c.n_pixels for c in wl.cameras)
    dl_all = torch.randn((P, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    _store_vs_replay(R, ps, wl.cameras, cfg, dl_all * 1e-3)
