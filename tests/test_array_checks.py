"""The Python binding checks every array it hands to the library (CPU): dtype,
layout, size against the scene description, and device.  The C ABI takes plain
pointers, so these checks are what keeps a wrong-sized tensor from turning into
out-of-bounds device accesses."""
import copy

import pytest
import torch

from paper_2510_08491_gb300 import _lib as L
from paper_2510_08491_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _scene(n=10, color=L.COLOR_SH, n_c=0, dynamic=False, bf16=False):
    from paper_2510_08491_gb300.render import PackedScene
    offs, stride = L.net_layout(8, color, n_c, dynamic)
    d = L.SceneDesc(n, 8, color, n_c, L.BF16 if bf16 else L.F32, 30.0, int(dynamic))
    net = torch.zeros((n, stride), dtype=torch.bfloat16 if bf16 else torch.float32)
    return PackedScene(d, torch.zeros((n, L.GEOM_STRIDE)), net, offs, stride)


def _msg(fn):
    with pytest.raises(ValueError) as ei:
        fn()
    return str(ei.value)


def test_need_checks_dtype_layout_size_then_device():
    from paper_2510_08491_gb300.render import _need
    f32 = (torch.float32,)
    _need(None, 5, 3, f32, "x")                                   # absent arrays pass
    assert "dtype" in _msg(lambda: _need(torch.zeros(5, 3, dtype=torch.float64), 5, 3, f32, "x"))
    assert "contiguous" in _msg(lambda: _need(torch.zeros(3, 5).t(), 5, 3, f32, "x"))
    assert "columns" in _msg(lambda: _need(torch.zeros(5, 4), 5, 3, f32, "x"))
    assert "at least" in _msg(lambda: _need(torch.zeros(4, 3), 5, 3, f32, "x"))
    assert "at least" in _msg(lambda: _need(torch.zeros(14), 5, 3, f32, "x"))
    assert "CUDA" in _msg(lambda: _need(torch.zeros(5, 3), 5, 3, f32, "x"))   # right shape, host memory
    assert "CUDA" in _msg(lambda: _need(torch.zeros(5, 2, 3), 5, 6, f32, "x"))  # any shape with enough elements
    assert "tensor" in _msg(lambda: _need([0.0] * 15, 5, 3, f32, "x"))


@pytest.mark.parametrize("kw", [{}, {"color": L.COLOR_MLP, "n_c": 32}, {"dynamic": True}, {"bf16": True}])
def test_packed_scene_is_checked_against_its_description(kw):
    ps = _scene(**kw)
    assert "CUDA" in _msg(ps.validate)            # consistent, but on the host
    bad = copy.copy(ps)
    bad.geom = ps.geom[:5]
    assert "geom" in _msg(bad.validate)
    bad = copy.copy(ps)
    bad.net = ps.net[:, :8].contiguous()
    assert "net" in _msg(bad.validate)
    bad = copy.copy(ps)
    bad.net = ps.net.float() if ps.net.dtype == torch.bfloat16 else ps.net.to(torch.bfloat16)
    assert "dtype" in _msg(bad.validate)
    bad = copy.copy(ps)
    bad.desc = L.SceneDesc.from_buffer_copy(ps.desc)
    bad.desc.n_sigma = 16                         # another layout than the arrays'
    assert "layout" in _msg(bad.validate)
    bad = copy.copy(ps)
    bad.desc = L.SceneDesc.from_buffer_copy(ps.desc)
    bad.desc.n = 11                               # more primitives than rows
    assert "at least" in _msg(bad.validate)
