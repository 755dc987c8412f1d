"""The synthetic workloads follow their stated recipes (CPU): the speed-protocol
scene uses the paper's primitive (N_sigma = 8, w0 = 30, four SH bands; Sec. 3.3)
and its initialisation of the density weights (W1 ~ U(-1/3, 1/3),
w2 ~ U(-sqrt(6/N_sigma)/w0, +)), square 800 x 800 views at a 39.6 degree field of
view; the dynamic variant gives view k the timestamp k / 7; generation is
deterministic for a seed."""
import math

import numpy as np

from paper_2510_08491_gb300 import synth


def test_speed_protocol_scene_and_cameras():
    wl = synth.workload("fps100k_800px_sh")
    sc = wl.scene
    assert (sc.n, sc.n_sigma, sc.omega0, sc.color) == (100_000, 8, 30.0, "sh")
    assert sc.sh.shape == (100_000, 16, 3)
    assert np.abs(sc.W1).max() <= 1.0 / 3.0 and np.abs(sc.W1).max() > 0.33
    lim = math.sqrt(6.0 / 8) / 30.0
    assert np.abs(sc.w2).max() <= lim and np.abs(sc.w2).max() > 0.99 * lim
    # uniform: mean near 0, variance near lim^2 / 3
    assert abs(sc.w2.mean()) < 0.01 * lim and abs(sc.w2.var() / (lim * lim / 3) - 1) < 0.01
    assert len(wl.cameras) == 8
    for c in wl.cameras:
        assert (c.width, c.height) == (800, 800)
        fov = 2 * math.degrees(math.atan((c.height / 2) / float(c.fy)))
        assert abs(fov - 39.6) < 1e-3
        assert abs(np.linalg.norm(c.eye) - 4.0) < 1e-4
    # the paper's 41 + 10 + 48 = 99 parameters per primitive
    dens = sc.W1[0].size + sc.b1[0].size + sc.w2[0].size + 1
    assert dens == 41 and dens + 10 + sc.sh[0].size == 99


def test_dynamic_variant_timestamps_and_determinism():
    a = synth.workload("dyn100k_800px_8t")
    assert a.scene.dynamic and a.scene.wt.shape == (100_000, 8) and a.scene.sh_t.shape == (100_000, 12, 3)
    assert [float(c.time) for c in a.cameras] == [float(np.float32(k / 7.0)) for k in range(8)]
    b = synth.workload("dyn100k_800px_8t")
    for f in a.scene.fields():
        assert np.array_equal(getattr(a.scene, f), getattr(b.scene, f)), f
    # the static scene is the dynamic one without its time fields (same draws before them)
    st = synth.workload("fps100k_800px_sh").scene
    for f in st.fields():
        assert np.array_equal(getattr(st, f), getattr(a.scene, f)), f
