"""GPU checks of the batched form: tile sizes 8/16/32, the length-ordered
persistent launches over many views of uneven size, CUDA-graph capture of the
whole forward + backward with reserved capacity, the capacity overflow report,
and the autotuner.
"""
import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth
from gpu_util import assert_image_close, grad_rel_errors, oracle_images, sample_tiles, tile_subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _uneven_views(n, radius, seed=0):
    g = np.random.default_rng(seed)
    res = [synth.RESOLUTIONS[i] for i in g.integers(0, 4, size=n)]
    res = [(w // 4, h // 4) for (w, h) in res]  # a quarter of the batched workload's sizes
    return synth.fibonacci_cameras(n, radius, res)


@pytest.mark.parametrize("color", ["const", "mlp"])
def test_tile_sizes_give_identical_images(R, oracle_lib, color):
    """The per-pixel work does not depend on the tiling: images are bit-identical
    for 8, 16 and 32 pixel tiles, and keys match the oracle for each tile size."""
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    O = oracle_lib
    sc = synth.make_scene(2500, seed=31, center_half=2.0, n_sigma=16, color=color, n_c=32)
    cams = _uneven_views(5, 7.0)
    ps = pack_scene(sc)
    imgs = {}
    for ts in (8, 16, 32):
        img = R.forward(ps, cams, L.make_config(tile_size=ts)).cpu().numpy()
        keys, vals = R.debug_keys()
        tl = O.tile_keys(sc, cams, ts)
        assert np.array_equal(keys, tl.keys) and np.array_equal(vals, tl.vals), ts
        imgs[ts] = img
    assert np.array_equal(imgs[8], imgs[16]) and np.array_equal(imgs[32], imgs[16])
    ref, flags, _, _ = oracle_images(O, sc, cams)
    assert_image_close(imgs[16], ref, flags)


@pytest.mark.parametrize("ts,nc", [(8, 32), (32, 32), (8, 64)])
def test_tile_size_backward(R, oracle_lib, ts, nc):
    """Backward at 8- and 32-pixel tiles against the oracle; at 8-pixel tiles and
    N_c = 64 the kernel accumulates dL/dWc2 with shared-memory atomics (not in
    tensor memory) and its flush permutes the 64 x 64 block from fragment order."""
    from test_gpu_backward import _check, _dl, _gpu_grads_cfg, _oracle_grads
    O = oracle_lib
    sc = synth.make_scene(1200, seed=3, center_half=1.5, n_sigma=16, omega0=5.0, color="mlp", n_c=nc)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 72, 56)]
    dLv = _dl(O, sc, cams, 3)
    g = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv), tile_size=ts)
    gref = _oracle_grads(O, sc, cams, dLv)
    _check(g, gref, sc.fields()[:3] + ["W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"])


def test_uneven_views_bf16_mlp64(R, oracle_lib):
    """16 views of uneven size, N_sigma = 32, N_c = 64, BF16 weights (the batched
    workload's shapes on a smaller scene): keys bit-exact, images within 1e-4."""
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    O = oracle_lib
    sc = synth.make_scene(6000, seed=41, center_half=3.0, n_sigma=32, color="mlp", n_c=64).to_bf16()
    cams = _uneven_views(16, 10.0, seed=7)
    ps = pack_scene(sc)
    img = R.forward(ps, cams, L.make_config()).cpu().numpy()
    keys, vals = R.debug_keys()
    ref, flags, tl, _ = oracle_images(O, sc, cams)
    assert np.array_equal(keys, tl.keys) and np.array_equal(vals, tl.vals)
    assert_image_close(img, ref, flags)


def test_graph_capture_matches_eager(R):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import GraphStep, Renderer, pack_scene
    sc = synth.make_scene(3000, seed=51, center_half=2.0, n_sigma=16, color="mlp", n_c=32)
    cams = _uneven_views(4, 7.0, seed=3)
    r = Renderer(0)
    ps = pack_scene(sc)
    cfg = L.make_config()
    P = r.image_size(cams)
    dL = torch.randn((P, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    img0 = r.forward(ps, cams, cfg).clone()
    gg0 = torch.zeros_like(ps.geom)
    gn0 = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
    r.backward(ps, dL, gg0, gn0)
    torch.cuda.synchronize()
    K = r.stats().n_keys
    step = GraphStep(r, ps, cams, cfg, max_keys=K + 1024, dL=dL)
    for _ in range(2):
        step.image.zero_()
        step.replay()
        torch.cuda.synchronize()
        assert torch.equal(step.image, img0)
        for a, b in ((step.g_geom, gg0), (step.g_net, gn0)):
            err = (a - b).abs().max().item()
            assert err <= 1e-5 * (b.abs().max().item() + 1e-12), err
    assert r.stats().n_keys == K


def test_graph_step_matches_oracle_bf16_mlp64_16views(R, oracle_lib):
    """The batched workload's form checked against the FP64 oracle: 16 views of
    uneven size, N_sigma = 32, N_c = 64, BF16 weights, 16-pixel tiles, forward chunk 3
    and the backward's default chunk (4 entries: the configuration the benchmark's
    autotuner settles on, tensor-memory dL/dWc2), forward + backward
    captured in one CUDA graph and replayed twice.  dL/dC is set on three sampled
    tiles per view (zero on termination near-ties and colour-MLP ReLU kinks); the
    image there and every gradient group must meet the parity bars against the
    oracle on the primitives those tiles list, and every other primitive's
    gradient must be exactly zero."""
    from oracle import grad as G
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import GraphStep, Renderer, pack_scene, unpack_geom_grad, unpack_net_grad
    from test_gpu_backward import GRAD_TOL, RELU_EPS
    O = oracle_lib
    sc = synth.make_scene(6000, seed=41, center_half=3.0, n_sigma=32, color="mlp", n_c=64).to_bf16()
    cams = _uneven_views(16, 10.0, seed=7)
    tl = O.tile_keys(sc, cams, 16)
    picks = sample_tiles(cams, tl, 16, 3, seed=43)
    sub, prims, per_view = tile_subset(O, sc, tl, picks)
    pix_off = np.concatenate([[0], np.cumsum([c.n_pixels for c in cams])])
    rng = np.random.default_rng(44)
    dL = np.zeros((int(pix_off[-1]), 3), np.float32)
    ref_rgb, gref = {}, None
    for v, (pix, owner, off, lst) in sorted(per_view.items()):
        out = O.render_pixels(sub, cams[v], pix, owner, off, lst)
        d = rng.normal(size=(len(pix), 3))
        d[out.flags != 0] = 0.0
        _, _, ah, amin = G.pair_diagnostics(sub, cams[v], pix, owner, off, lst)
        pair_pix = np.repeat(np.arange(len(pix)), off[owner + 1] - off[owner])
        d[np.unique(pair_pix[(ah > 0) & (amin < RELU_EPS)])] = 0.0
        dL[pix_off[v] + pix] = d
        ref_rgb[v] = out
        _, g = G.grads(sub, cams[v], pix, owner, off, lst, d)
        gref = g if gref is None else {k: gref[k] + g[k] for k in g}
    r = Renderer(0)
    ps = pack_scene(sc)
    cfg = L.make_config(tile_size=16, chunk=3)
    r.forward(ps, cams, cfg)
    K = r.stats().n_keys
    step = GraphStep(r, ps, cams, cfg, max_keys=K + 4096, dL=torch.tensor(dL, device="cuda"))
    fields = ["centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3",
              "bc3"]
    others = np.ones(sc.n, bool)
    others[prims] = False
    for _ in range(2):
        step.image.zero_()
        step.replay()
        torch.cuda.synchronize()
        img = step.image.cpu().numpy()
        for v, (pix, owner, off, lst) in per_view.items():
            assert_image_close(img[pix_off[v] + pix], ref_rgb[v].rgb, ref_rgb[v].flags)
        g = unpack_geom_grad(step.g_geom)
        g.update(unpack_net_grad(ps, step.g_net, sc))
        for f in fields:
            assert not np.any(g[f][others]), f
        errs = grad_rel_errors({f: g[f][prims] for f in fields}, {f: gref[f] for f in fields})
        print({k: (f"{a:.1e}", f"{b:.1e}") for k, (a, b) in errs.items()})
        bad = {k: e for k, e in errs.items() if e[0] > GRAD_TOL or e[1] > GRAD_TOL}
        assert not bad, bad
    assert r.stats().n_keys == K


def test_two_graphs_share_a_reservation(R):
    """Two captured steps over different scenes and outputs on one reservation,
    replayed alternately, each reproduce their eager result."""
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import GraphStep, Renderer, pack_scene
    sc = synth.make_scene(2500, seed=52, center_half=2.0, n_sigma=16, color="mlp", n_c=32)
    sc2 = synth.perturb(sc, seed=53, std=0.02)
    cams = _uneven_views(3, 7.0, seed=4)
    r = Renderer(0)
    cfg = L.make_config()
    P = r.image_size(cams)
    dL = torch.randn((P, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    eager, pss = [], []
    for s_ in (sc, sc2):
        ps = pack_scene(s_)
        img = r.forward(ps, cams, cfg).clone()
        gg = torch.zeros_like(ps.geom)
        gn = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
        r.backward(ps, dL, gg, gn)
        eager.append((img, gg, gn))
        pss.append(ps)
    torch.cuda.synchronize()
    K = max(r.stats().n_keys, 1)
    steps = [GraphStep(r, pss[0], cams, cfg, max_keys=2 * K + 4096, dL=dL),
             GraphStep(r, pss[1], cams, cfg, max_keys=0, dL=dL, reserve=False)]
    for _ in range(2):
        for st, (img, gg, gn) in zip(steps, eager):
            st.replay()
            torch.cuda.synchronize()
            assert torch.equal(st.image, img)
            for a, b in ((st.g_geom, gg), (st.g_net, gn)):
                assert (a - b).abs().max().item() <= 1e-5 * (b.abs().max().item() + 1e-12)


def test_capacity_overflow_is_reported(R):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import Renderer, pack_scene
    sc = synth.make_scene(2000, seed=61, center_half=2.0, n_sigma=8)
    cams = synth.ring_cameras(2, 6.0, 160, 120)
    r = Renderer(0)
    ps = pack_scene(sc)
    cfg = L.make_config()
    r.reserve(ps, cams, cfg, max_keys=100)
    r.forward(ps, cams, cfg)  # reserved: no growth, keys beyond capacity are dropped and flagged
    with pytest.raises(L.SnpError) as ei:
        r.stats()
    assert ei.value.status == L.SNP_ERR_CAPACITY


def test_autotune_picks_a_working_configuration(R, tmp_path):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    sc = synth.make_scene(4000, seed=71, center_half=2.0, n_sigma=16, color="mlp", n_c=32)
    cams = _uneven_views(3, 7.0, seed=9)
    ps = pack_scene(sc)
    cache = str(tmp_path / "tune.json")
    best = R.autotune(ps, cams, L.make_config(), backward=True, cache_path=cache)
    assert best.tile_size in (8, 16, 32) and best.chunk >= 1
    again = R.autotune(ps, cams, L.make_config(), backward=True, cache_path=cache)
    assert (again.tile_size, again.chunk) == (best.tile_size, best.chunk)
    img = R.forward(ps, cams, best).cpu().numpy()
    ref = R.forward(ps, cams, L.make_config()).cpu().numpy()
    assert np.array_equal(img, ref)


def test_reserved_context_rejects_another_tile_size(R):
    """A reservation fixes the tile size (the composited masks and key capacity are
    sized for it): a forward with another tile size is refused, not overrun."""
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import Renderer, pack_scene
    sc = synth.make_scene(500, seed=81, center_half=1.5, n_sigma=8)
    cams = synth.ring_cameras(1, 6.0, 96, 64)
    r = Renderer(0)
    ps = pack_scene(sc)
    r.reserve(ps, cams, L.make_config(tile_size=16))
    with pytest.raises(L.SnpError) as ei:
        r.forward(ps, cams, L.make_config(tile_size=32))
    assert ei.value.status == L.SNP_ERR_INVALID_ARG
    img = r.forward(ps, cams, L.make_config(tile_size=16))
    assert torch.isfinite(img).all()


def test_reserve_rejects_32bit_index_overflow(R):
    """The key value v * n + i and the key offsets are 32-bit: a reservation for more
    than 2^32 - 1 instances or keys is refused before any allocation or launch, and
    leaves the context usable."""
    import copy
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import Renderer, pack_scene
    sc = synth.make_scene(300, seed=91, center_half=1.5, n_sigma=8)
    r = Renderer(0)
    ps = pack_scene(sc)
    big = copy.copy(ps)
    big.desc = L.SceneDesc.from_buffer_copy(ps.desc)
    big.desc.n = 1 << 27
    cams33 = synth.ring_cameras(33, 6.0, 16, 16)   # 33 * 2^27 > 2^32 - 1
    with pytest.raises(L.SnpError) as ei:
        r.reserve(big, cams33, L.make_config())
    assert ei.value.status == L.SNP_ERR_UNSUPPORTED
    cams = synth.ring_cameras(1, 6.0, 96, 64)
    with pytest.raises(L.SnpError) as ei:
        r.reserve(ps, cams, L.make_config(), max_keys=1 << 32)
    assert ei.value.status == L.SNP_ERR_UNSUPPORTED
    img = r.forward(ps, cams, L.make_config())
    ref = R.forward(ps, cams, L.make_config())
    assert torch.equal(img, ref)


def test_backward_refuses_a_description_other_than_the_forwards(R):
    """The backward replays the forward's lists with the forward's layout: a scene
    description that differs from the forward's (here only in omega0, which changes
    no array size) is refused before any launch."""
    import copy
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import Renderer, pack_scene
    sc = synth.make_scene(300, seed=93, center_half=1.5, n_sigma=8)
    cams = synth.ring_cameras(1, 6.0, 96, 64)
    r = Renderer(0)
    ps = pack_scene(sc)
    img = r.forward(ps, cams, L.make_config())
    other = copy.copy(ps)
    other.desc = L.SceneDesc.from_buffer_copy(ps.desc)
    other.desc.omega0 = float(ps.desc.omega0) * 2.0
    g_geom = torch.zeros_like(ps.geom)
    with pytest.raises(L.SnpError) as ei:
        r.backward(other, torch.ones_like(img), g_geom, None)
    assert ei.value.status == L.SNP_ERR_INVALID_ARG
    assert not torch.any(g_geom)
    r.backward(ps, torch.ones_like(img), g_geom, None)
    torch.cuda.synchronize()
    assert torch.isfinite(g_geom).all() and torch.any(g_geom)


def test_wrong_sized_arrays_are_refused_before_any_launch(R):
    """The binding checks array sizes against the scene description (the ABI sees
    only pointers).  The short arrays here are views of full-size allocations, so
    nothing could be read out of bounds even without the check."""
    import copy
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    sc = synth.make_scene(300, seed=95, center_half=1.5, n_sigma=8)
    cams = synth.ring_cameras(1, 6.0, 96, 64)
    ps = pack_scene(sc)
    bad = copy.copy(ps)
    bad.geom = ps.geom[:200]
    n0 = L.kernel_launches()
    with pytest.raises(ValueError):
        R.forward(bad, cams, L.make_config())
    assert L.kernel_launches() == n0
    img = R.forward(ps, cams, L.make_config())
    g_geom = torch.zeros_like(ps.geom)
    n1 = L.kernel_launches()
    with pytest.raises(ValueError):
        R.backward(ps, img[:100], g_geom, None)
    with pytest.raises(ValueError):
        R.backward(ps, torch.ones_like(img), g_geom[:200], None)
    assert L.kernel_launches() == n1
    assert not torch.any(g_geom)
