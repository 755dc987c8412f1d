"""PyTorch-facing renderer: device tensors in, images (and gradients) out, through libsnp.

PyTorch provides device memory and streams only; projection, sorting,
rasterisation and the backward all run in the CUDA library.  There is no CPU
or PyTorch fallback: without a built libsnp.so and a CUDA device every entry
point raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L

NET_FIELDS = ("W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3")


@dataclass
class PackedScene:
    """Device arrays in the library's layout plus their description."""

    desc: L.SceneDesc
    geom: torch.Tensor  # float32 [n, 16]
    net: torch.Tensor  # [n, stride] float32 or bfloat16
    offsets: List[int]
    stride: int

    @property
    def n(self) -> int:
        return int(self.desc.n)

    def ptrs(self) -> L.ScenePtrs:
        return L.ScenePtrs(self.geom.data_ptr() if self.n else None, self.net.data_ptr() if self.n else None)


def pack_scene(scene, device="cuda", weight_dtype: Optional[str] = None) -> PackedScene:
    """Lay a synth.Scene out as the library's geometry [n, 16] and network [n, stride] arrays."""
    wd = weight_dtype or scene.weight_dtype
    mlp = scene.color == "mlp"
    cm = L.COLOR_MLP if mlp else L.COLOR_CONST
    offs, stride = L.net_layout(scene.n_sigma, cm, scene.n_c)
    n = scene.n
    geom = np.zeros((n, L.GEOM_STRIDE), np.float32)
    geom[:, 0:3] = scene.centers
    geom[:, 3:6] = scene.log_scales
    geom[:, 6:10] = scene.quats
    geom[:, 10:13] = scene.rgb
    net = np.zeros((n, stride), np.float32)
    for k, f in enumerate(NET_FIELDS):
        if offs[k] < 0:
            continue
        a = getattr(scene, f)
        a = a.reshape(n, int(np.prod(a.shape[1:])) if a.ndim > 1 else 1)
        net[:, offs[k]:offs[k] + a.shape[1]] = a
    desc = L.SceneDesc(n, scene.n_sigma, cm, scene.n_c if mlp else 0, L.BF16 if wd == "bf16" else L.F32,
                       float(scene.omega0), 0)
    g = torch.from_numpy(geom).to(device)
    t = torch.from_numpy(net).to(device)
    if wd == "bf16":
        t = t.to(torch.bfloat16)  # exact for values already rounded to bf16
    return PackedScene(desc, g.contiguous(), t.contiguous(), offs, stride)


def unpack_net_grad(ps: PackedScene, g_net: torch.Tensor, scene) -> dict:
    """Split a [n, stride] gradient into the named parameter arrays (numpy, float64)."""
    out = {}
    g = g_net.double().cpu().numpy()
    for k, f in enumerate(NET_FIELDS):
        if ps.offsets[k] < 0:
            continue
        shp = getattr(scene, f).shape
        size = int(np.prod(shp[1:])) if len(shp) > 1 else 1
        out[f] = g[:, ps.offsets[k]:ps.offsets[k] + size].reshape(shp)
    return out


def unpack_geom_grad(g_geom: torch.Tensor) -> dict:
    g = g_geom.double().cpu().numpy()
    return {"centers": g[:, 0:3], "log_scales": g[:, 3:6], "quats": g[:, 6:10], "rgb": g[:, 10:13]}


class Renderer:
    """One libsnp context plus the stream-level calls."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the snp renderer needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.ctx = L.Context(device)
        self.token = 0

    def image_size(self, cams) -> int:
        return sum(c.width * c.height for c in cams)

    def forward(self, ps: PackedScene, cams, cfg: Optional[L.Config] = None, out: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        cfg = cfg or L.make_config()
        carr = L.make_cameras(cams)
        P = self.image_size(cams)
        if out is None:
            out = torch.empty((P, 3), dtype=torch.float32, device=self.device)
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        tok = C.c_int64()
        sp = ps.ptrs()
        self.ctx.check(L.lib().snp_render_forward(self.ctx.handle, C.byref(ps.desc), C.byref(sp), carr, len(cams),
                                                  C.byref(cfg), C.c_void_p(out.data_ptr()), C.byref(tok),
                                                  C.c_void_p(st)))
        self.token = tok.value
        return out

    def backward(self, ps: PackedScene, dL: torch.Tensor, g_geom: Optional[torch.Tensor],
                 g_net: Optional[torch.Tensor], token: Optional[int] = None,
                 stream: Optional[torch.cuda.Stream] = None):
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        gp = L.GradPtrs(g_geom.data_ptr() if g_geom is not None else None,
                        g_net.data_ptr() if g_net is not None else None)
        sp = ps.ptrs()
        self.ctx.check(L.lib().snp_render_backward(self.ctx.handle, int(token or self.token), C.byref(ps.desc),
                                                   C.byref(sp), C.c_void_p(dL.contiguous().data_ptr()),
                                                   C.byref(gp), C.c_void_p(st)))

    def stats(self, token: Optional[int] = None) -> L.Stats:
        s = L.Stats()
        st = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx.check(L.lib().snp_get_stats(self.ctx.handle, int(token or self.token), C.byref(s), C.c_void_p(st)))
        return s

    def debug_keys(self, token: Optional[int] = None):
        st = torch.cuda.current_stream(self.device).cuda_stream
        k = C.c_int64()
        self.ctx.check(L.lib().snp_debug_keys(self.ctx.handle, int(token or self.token), None, None, 0,
                                              C.byref(k), C.c_void_p(st)))
        K = k.value
        keys = np.zeros(K, np.uint64)
        vals = np.zeros(K, np.uint32)
        self.ctx.check(L.lib().snp_debug_keys(self.ctx.handle, int(token or self.token),
                                              keys.ctypes.data_as(C.c_void_p), vals.ctypes.data_as(C.c_void_p),
                                              K, C.byref(k), C.c_void_p(st)))
        return keys, vals

    def reserve(self, ps: PackedScene, cams, cfg: Optional[L.Config] = None, max_keys: int = 0):
        cfg = cfg or L.make_config()
        carr = L.make_cameras(cams)
        self.ctx.check(L.lib().snp_reserve(self.ctx.handle, C.byref(ps.desc), carr, len(cams), C.byref(cfg),
                                           int(max_keys)))


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, geom, net, renderer, ps, cams, cfg):
        img = renderer.forward(ps, cams, cfg)
        ctx.renderer, ctx.ps, ctx.token = renderer, ps, renderer.token
        return img

    @staticmethod
    def backward(ctx, dL):
        r, ps = ctx.renderer, ctx.ps
        g_geom = torch.zeros_like(ps.geom) if ctx.needs_input_grad[0] else None
        need_net = ctx.needs_input_grad[1]
        g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device=ps.net.device) if need_net else None
        r.backward(ps, dL.contiguous(), g_geom, g_net, ctx.token)
        if g_net is not None and ps.net.dtype != torch.float32:
            g_net = g_net.to(ps.net.dtype)
        return g_geom, g_net, None, None, None, None


def render(renderer: Renderer, ps: PackedScene, cams, cfg: Optional[L.Config] = None) -> torch.Tensor:
    """Differentiable render: images [sum H*W, 3] (views concatenated, HWC) as a function of
    ps.geom and ps.net (set requires_grad on them to get gradients)."""
    return _RenderFn.apply(ps.geom, ps.net, renderer, ps, cams, cfg or L.make_config())
