"""Resident CTAs per SM of the persistent raster launches, as the library reports
them (snp_stats.fwd_ctas_per_sm / bwd_ctas_per_sm).

A default chunk is the largest whose shared memory keeps the CTAs per SM that the
kernel is built for (its __launch_bounds__ minimum): three forward and two
backward CTAs at 16-pixel tiles with a colour network at most 32 wide or none,
two forward and one backward CTA at N_c = 64.  A chunk whose dynamic shared
memory plus the kernel's static shared memory and the per-CTA reservation no
longer fits that many CTAs still runs, one CTA per SM fewer and much slower, so
this checks the count the launches actually got, for every colour mode, the
time-conditioned scenes and several N_sigma.
"""
import pytest
import torch

from paper_2510_08491_gb300 import synth

pytestmark = pytest.mark.gpu

# (colour, n_sigma, n_c, bf16, dynamic) -> CTAs per SM of the forward, backward
CASES = [
    (("mlp", 16, 32, False, False), (3, 2)),
    (("mlp", 32, 32, False, False), (3, 2)),
    (("mlp", 32, 64, True, False), (2, 1)),
    (("sh", 8, 0, False, False), (3, 2)),
    (("sh", 16, 0, False, False), (3, 2)),
    (("sh", 8, 0, False, True), (3, 2)),
    (("const", 16, 0, False, False), (3, 2)),
    (("const", 32, 0, True, True), (3, 2)),
]


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


@pytest.mark.parametrize("case,expect", CASES, ids=lambda c: "-".join(str(x) for x in c))
def test_default_chunks_keep_the_designed_ctas_per_sm(R, case, expect):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    color, ns, nc, bf16, dyn = case
    sc = synth.make_scene(1500, seed=5, center_half=2.0, n_sigma=ns, omega0=10.0, color=color, n_c=nc, dynamic=dyn)
    if bf16:
        sc = sc.to_bf16()
    cams = synth.ring_cameras(2, 7.0, 96, 80)
    ps = pack_scene(sc)
    img = R.forward(ps, cams, L.make_config())
    dL = torch.full_like(img, 1e-3)
    g_geom = torch.zeros_like(ps.geom)
    g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
    R.backward(ps, dL, g_geom, g_net)
    torch.cuda.synchronize()
    st = R.stats()
    d = ps.desc
    chunks = L.default_chunks(int(d.n_sigma), int(d.color_mode), int(d.n_c), 16, bool(d.dynamic))
    assert (st.fwd_ctas_per_sm, st.bwd_ctas_per_sm) == expect, \
        f"{case}: default chunks {chunks} ran {st.fwd_ctas_per_sm} / {st.bwd_ctas_per_sm} CTAs per SM"
