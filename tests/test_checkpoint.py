"""Scene files and training checkpoints (CPU): a scene written by
synth.save_scene reads back field for field (cameras included) and renders the
same image in the oracle; a packed scene plus optimiser state written by
render.save_checkpoint reads back bit for bit, BF16 networks included."""
import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth


@pytest.mark.parametrize("color,dynamic", [("const", False), ("mlp", False), ("sh", True)])
def test_scene_file_round_trip(tmp_path, oracle_lib, color, dynamic):
    O = oracle_lib
    sc = synth.make_scene(40, seed=3, center_half=1.0, n_sigma=8, omega0=5.0, color=color, n_c=32,
                          dynamic=dynamic)
    cams = synth.ring_cameras(2, 4.0, 40, 32)
    cams[1].time = np.float32(0.4)
    path = str(tmp_path / "scene.npz")
    synth.save_scene(sc, path, cams)
    sc2, cams2 = synth.load_scene(path)
    assert sc2.fields() == sc.fields()
    for f in sc.fields():
        assert np.array_equal(getattr(sc2, f), getattr(sc, f)), f
    for a, b in zip(cams, cams2):
        assert np.array_equal(a.R_wc, b.R_wc) and np.array_equal(a.eye, b.eye)
        assert (a.width, a.height, a.fx, a.cx, a.time) == (b.width, b.height, b.fx, b.cx, b.time)
    # the oracle reads the same file
    for v in range(2):
        i1 = O.render_view_brute(sc, cams[v], t_min=0.0).rgb
        i2 = O.render_view_brute(sc2, cams2[v], t_min=0.0).rgb
        assert np.array_equal(i1, i2)


@pytest.mark.parametrize("bf16", [False, True])
def test_checkpoint_round_trip(tmp_path, bf16):
    from paper_2510_08491_gb300 import build
    build.build()  # the layout comes from the library (loads without a GPU)
    from paper_2510_08491_gb300.render import load_checkpoint, pack_scene, save_checkpoint
    sc = synth.make_scene(50, seed=4, n_sigma=8, color="mlp", n_c=32)
    if bf16:
        sc = sc.to_bf16()
    ps = pack_scene(sc, device="cpu")
    state = {"m_net": torch.randn(ps.net.shape), "v_geom": torch.rand(ps.geom.shape)}
    path = str(tmp_path / "ckpt.npz")
    save_checkpoint(path, ps, state, step=17)
    ps2, state2, step = load_checkpoint(path, device="cpu")
    assert step == 17
    assert torch.equal(ps2.geom, ps.geom) and ps2.net.dtype == ps.net.dtype and torch.equal(ps2.net, ps.net)
    assert ps2.offsets == ps.offsets and ps2.stride == ps.stride
    for f in ("n", "n_sigma", "color_mode", "n_c", "weight_dtype", "omega0", "dynamic"):
        assert getattr(ps2.desc, f) == getattr(ps.desc, f)
    for k, t in state.items():
        assert torch.equal(state2[k], t)
