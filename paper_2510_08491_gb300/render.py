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

NET_FIELDS = ("W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3", "sh", "wt", "sh_t")


def _need(t: Optional[torch.Tensor], rows: int, cols: int, dtypes, name: str, device: bool = True) -> None:
    """Check an array handed to the library: on the GPU, contiguous, of one of
    `dtypes`, at least `rows` rows of `cols` elements (a 2-D tensor must have exactly
    `cols` columns).  The C ABI takes plain pointers and cannot see sizes, so a
    mismatch would otherwise become out-of-bounds device accesses.  None passes."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: dtype {t.dtype}, expected one of {tuple(dtypes)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.dim() == 2 and t.shape[1] != cols:
        raise ValueError(f"{name}: {t.shape[1]} columns, expected {cols}")
    if t.numel() < rows * cols:
        raise ValueError(f"{name}: {t.numel()} elements, expected at least {rows} x {cols}")
    if device and not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")


_F32 = (torch.float32,)
_I32 = (torch.int32,)


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

    def validate(self) -> None:
        """Raise ValueError unless the arrays match the description: geometry float32
        [n, 16], network [n, stride] in the description's weight type and layout."""
        d = self.desc
        offs, stride = L.net_layout(int(d.n_sigma), int(d.color_mode), int(d.n_c), bool(d.dynamic))
        if stride != self.stride or list(offs) != list(self.offsets):
            raise ValueError("network layout differs from the scene description's")
        _need(self.geom, self.n, L.GEOM_STRIDE, _F32, "geom", device=False)
        _need(self.net, self.n, stride, (torch.bfloat16,) if d.weight_dtype == L.BF16 else _F32, "net", device=False)
        for t, name in ((self.geom, "geom"), (self.net, "net")):
            if not t.is_cuda:
                raise ValueError(f"{name}: expected a CUDA tensor")


def pack_scene(scene, device="cuda", weight_dtype: Optional[str] = None) -> PackedScene:
    """Lay a synth.Scene out as the library's geometry [n, 16] and network [n, stride] arrays."""
    wd = weight_dtype or scene.weight_dtype
    mlp = scene.color == "mlp"
    cm = {"const": L.COLOR_CONST, "mlp": L.COLOR_MLP, "sh": L.COLOR_SH}[scene.color]
    dyn = bool(getattr(scene, "dynamic", False))
    offs, stride = L.net_layout(scene.n_sigma, cm, scene.n_c, dyn)
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
                       float(scene.omega0), int(dyn))
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


_DESC_FIELDS = ("n", "n_sigma", "color_mode", "n_c", "weight_dtype", "omega0", "dynamic")


def save_checkpoint(path: str, ps: PackedScene, state: Optional[dict] = None, step: int = 0) -> None:
    """Write the packed scene (geometry and network arrays in the library's layout),
    optional optimiser state (name -> tensor, e.g. Adam moments and an FP32 master
    copy) and the step count to one .npz file.  BF16 networks keep their exact bits."""
    arrays = {"geom": ps.geom.detach().cpu().numpy()}
    if ps.net.dtype == torch.bfloat16:
        arrays["net_bf16_bits"] = ps.net.detach().cpu().view(torch.int16).numpy()
    else:
        arrays["net"] = ps.net.detach().cpu().numpy()
    for k, t in (state or {}).items():
        arrays["state_" + k] = t.detach().cpu().numpy()
    desc = np.asarray([float(getattr(ps.desc, f)) for f in _DESC_FIELDS], np.float64)
    np.savez(path, desc=desc, offsets=np.asarray(ps.offsets, np.int32), stride=np.int32(ps.stride),
             step=np.int64(step), **arrays)


def load_checkpoint(path: str, device="cuda"):
    """Read a file written by save_checkpoint: returns (PackedScene, state dict, step)."""
    z = np.load(path)
    d = z["desc"]
    desc = L.SceneDesc(int(d[0]), int(d[1]), int(d[2]), int(d[3]), int(d[4]), float(d[5]), int(d[6]))
    geom = torch.from_numpy(z["geom"]).to(device)
    if "net_bf16_bits" in z:
        net = torch.from_numpy(z["net_bf16_bits"]).view(torch.bfloat16).to(device)
    else:
        net = torch.from_numpy(z["net"]).to(device)
    state = {k[len("state_"):]: torch.from_numpy(z[k]).to(device) for k in z.files if k.startswith("state_")}
    ps = PackedScene(desc, geom.contiguous(), net.contiguous(), [int(x) for x in z["offsets"]], int(z["stride"]))
    return ps, state, int(z["step"])


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
        ps.validate()
        carr = L.make_cameras(cams)
        P = self.image_size(cams)
        if out is None:
            out = torch.empty((P, 3), dtype=torch.float32, device=self.device)
        _need(out, P, 3, _F32, "out")
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        tok = C.c_int64()
        sp = ps.ptrs()
        self.ctx.check(L.lib().snp_render_forward(self.ctx.handle, C.byref(ps.desc), C.byref(sp), carr, len(cams),
                                                  C.byref(cfg), C.c_void_p(out.data_ptr()), C.byref(tok),
                                                  C.c_void_p(st)))
        self.token = tok.value
        self._pixels = P
        return out

    def backward(self, ps: PackedScene, dL: torch.Tensor, g_geom: Optional[torch.Tensor],
                 g_net: Optional[torch.Tensor], token: Optional[int] = None,
                 stream: Optional[torch.cuda.Stream] = None):
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        ps.validate()
        dL = dL.contiguous()
        _need(dL, getattr(self, "_pixels", 0), 3, _F32, "dL")
        _need(g_geom, ps.n, L.GEOM_STRIDE, _F32, "g_geom")
        _need(g_net, ps.n, ps.stride, _F32, "g_net")
        gp = L.GradPtrs(g_geom.data_ptr() if g_geom is not None else None,
                        g_net.data_ptr() if g_net is not None else None)
        sp = ps.ptrs()
        self.ctx.check(L.lib().snp_render_backward(self.ctx.handle, int(token or self.token), C.byref(ps.desc),
                                                   C.byref(sp), C.c_void_p(dL.data_ptr()),
                                                   C.byref(gp), C.c_void_p(st)))

    def mse_loss(self, image: torch.Tensor, target: torch.Tensor, dL: Optional[torch.Tensor] = None,
                 loss: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None):
        """Mean squared error of image vs target and its gradient (snp_mse_loss), on the
        device and without synchronising: returns (loss [1] tensor, dL/dimage)."""
        if image.shape != target.shape or image.dtype != torch.float32 or target.dtype != torch.float32:
            raise ValueError("image and target must be float32 tensors of one shape")
        image, target = image.contiguous(), target.contiguous()
        dL = torch.empty_like(image) if dL is None else dL
        loss = torch.empty(1, dtype=torch.float32, device=image.device) if loss is None else loss
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        self.ctx.check(L.lib().snp_mse_loss(self.ctx.handle, C.c_void_p(image.data_ptr()),
                                            C.c_void_p(target.data_ptr()), image.numel(),
                                            C.c_void_p(dL.data_ptr()), C.c_void_p(loss.data_ptr()),
                                            C.c_void_p(st)))
        return loss, dL

    # ------------------------------------------------------------ training-step services

    def _st(self, stream=None) -> C.c_void_p:
        return C.c_void_p((stream or torch.cuda.current_stream(self.device)).cuda_stream)

    def popctl_accumulate(self, ps: PackedScene, g_net: torch.Tensor, stat_sum: torch.Tensor,
                          stat_count: torch.Tensor, stream=None):
        """Add this step's density-network gradient norm per primitive (snp_popctl_accumulate)."""
        ps.validate()
        _need(g_net, ps.n, ps.stride, _F32, "g_net")
        _need(stat_sum, ps.n, 1, _F32, "stat_sum")
        _need(stat_count, ps.n, 1, _I32, "stat_count")
        self.ctx.check(L.lib().snp_popctl_accumulate(self.ctx.handle, C.byref(ps.desc), C.c_void_p(g_net.data_ptr()),
                                                     C.c_void_p(stat_sum.data_ptr()),
                                                     C.c_void_p(stat_count.data_ptr()), self._st(stream)))

    def popctl_plan(self, ps: PackedScene, stat_sum: torch.Tensor, stat_count: torch.Tensor, cfg: L.PopctlConfig,
                    stream=None):
        """Per-primitive actions and output offsets (snp_popctl_plan); returns (action, offset, n_out)."""
        n = ps.n
        ps.validate()
        _need(stat_sum, n, 1, _F32, "stat_sum")
        _need(stat_count, n, 1, _I32, "stat_count")
        action = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        offset = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)  # uint32 bits
        n_out = C.c_int64(0)
        self.ctx.check(L.lib().snp_popctl_plan(self.ctx.handle, C.byref(ps.desc), C.c_void_p(ps.geom.data_ptr()),
                                               C.c_void_p(stat_sum.data_ptr()), C.c_void_p(stat_count.data_ptr()),
                                               C.byref(cfg), C.c_void_p(action.data_ptr()),
                                               C.c_void_p(offset.data_ptr()), C.byref(n_out), self._st(stream)))
        return action[:n], offset[:n], int(n_out.value)

    def popctl_apply(self, ps: PackedScene, action: torch.Tensor, offset: torch.Tensor, n_out: int,
                     noise: torch.Tensor, stream=None) -> PackedScene:
        """The new scene of a plan (snp_popctl_apply); noise is float32 [n, 2, 3] standard normal."""
        ps.validate()
        _need(action, ps.n, 1, _I32, "action")
        _need(offset, ps.n, 1, _I32, "offset")
        _need(noise, ps.n, 6, _F32, "noise")
        geom = torch.empty((max(n_out, 1), L.GEOM_STRIDE), dtype=torch.float32, device=self.device)
        net = torch.empty((max(n_out, 1), ps.stride), dtype=ps.net.dtype, device=self.device)
        self.ctx.check(L.lib().snp_popctl_apply(self.ctx.handle, C.byref(ps.desc), C.byref(ps.ptrs()),
                                                C.c_void_p(action.data_ptr()), C.c_void_p(offset.data_ptr()),
                                                C.c_void_p(noise.data_ptr()), C.c_void_p(geom.data_ptr()),
                                                C.c_void_p(net.data_ptr()), self._st(stream)))
        d = L.SceneDesc(n_out, ps.desc.n_sigma, ps.desc.color_mode, ps.desc.n_c, ps.desc.weight_dtype,
                        ps.desc.omega0, ps.desc.dynamic)
        return PackedScene(d, geom[:n_out], net[:n_out], ps.offsets, ps.stride)

    def geom_reg(self, ps: PackedScene, weight: float, g_geom: Optional[torch.Tensor],
                 loss: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Anisotropy regulariser (snp_geom_reg): returns the loss [1]; adds its gradient into g_geom."""
        loss = torch.empty(1, dtype=torch.float32, device=self.device) if loss is None else loss
        _need(ps.geom, ps.n, L.GEOM_STRIDE, _F32, "geom")
        _need(g_geom, ps.n, L.GEOM_STRIDE, _F32, "g_geom")
        _need(loss, 1, 1, _F32, "loss")
        self.ctx.check(L.lib().snp_geom_reg(self.ctx.handle, C.byref(ps.desc), C.c_void_p(ps.geom.data_ptr()),
                                            float(weight), C.c_void_p(g_geom.data_ptr() if g_geom is not None else None),
                                            C.c_void_p(loss.data_ptr()), self._st(stream)))
        return loss

    def adam_step(self, ps: PackedScene, g_geom, g_net, m_geom, v_geom, m_net, v_net, cfg: L.AdamConfig,
                  net_master: Optional[torch.Tensor] = None, stream=None):
        """One fused Adam step over the geometry and network arrays (snp_adam_step)."""
        def ptr(t):
            return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p()
        ps.validate()
        for t, name in ((g_geom, "g_geom"), (m_geom, "m_geom"), (v_geom, "v_geom")):
            _need(t, ps.n, L.GEOM_STRIDE, _F32, name)
        for t, name in ((g_net, "g_net"), (m_net, "m_net"), (v_net, "v_net"), (net_master, "net_master")):
            _need(t, ps.n, ps.stride, _F32, name)
        g = L.GradPtrs(g_geom.data_ptr() if g_geom is not None else None,
                       g_net.data_ptr() if g_net is not None else None)
        self.ctx.check(L.lib().snp_adam_step(self.ctx.handle, C.byref(ps.desc), ptr(ps.geom), ptr(ps.net),
                                             ptr(net_master), C.byref(g), ptr(m_geom), ptr(v_geom), ptr(m_net),
                                             ptr(v_net), C.byref(cfg), self._st(stream)))

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


    def autotune(self, ps: PackedScene, cams, cfg: Optional[L.Config] = None, backward: bool = True,
                 cache_path: Optional[str] = None) -> L.Config:
        """Pick tile size and staging chunk by timing them on this scene (snp_autotune).
        With cache_path, results are memoised in a JSON file keyed by GPU and shapes."""
        import json
        import os
        cfg = cfg or L.make_config()
        ps.validate()
        key = "|".join(str(x) for x in (torch.cuda.get_device_name(self.device), ps.n, ps.desc.n_sigma,
                                        ps.desc.color_mode, ps.desc.n_c, ps.desc.weight_dtype, ps.desc.dynamic,
                                        cfg.integral_form, int(backward), tuple((c.width, c.height) for c in cams)))
        cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    cache = json.load(f)
            except Exception:
                cache = {}
        if key in cache:
            best = L.make_config(tile_size=cache[key]["tile_size"], chunk=cache[key]["chunk"], form=cfg.integral_form,
                                 t_min=cfg.t_min, bg=tuple(cfg.bg), bwd_chunk=cfg.bwd_chunk)
            best.flags = cfg.flags
            return best
        best = L.Config()
        ms = C.c_float()
        st = torch.cuda.current_stream(self.device).cuda_stream
        sp = ps.ptrs()
        carr = L.make_cameras(cams)
        self.ctx.check(L.lib().snp_autotune(self.ctx.handle, C.byref(ps.desc), C.byref(sp), carr, len(cams),
                                            C.byref(cfg), int(backward), C.byref(best), C.byref(ms), C.c_void_p(st)))
        best.flags = cfg.flags
        if cache_path:
            cache[key] = {"tile_size": best.tile_size, "chunk": best.chunk, "ms": ms.value}
            tmp = cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, cache_path)
        self.last_autotune_ms = ms.value
        return best


class GraphStep:
    """Forward + backward of a fixed scene layout and camera set captured into one CUDA graph.

    The context reserves every workspace buffer first (no allocation and no host
    synchronisation inside the graph); the number of tile keys is bounded by
    max_keys and an overflow is reported by Renderer.stats().  Replay reads the
    current contents of ps.geom / ps.net and dL and writes image / grads."""

    def __init__(self, renderer: Renderer, ps: PackedScene, cams, cfg: L.Config, max_keys: int,
                 dL: Optional[torch.Tensor] = None, backward: bool = True, target: Optional[torch.Tensor] = None,
                 reserve: bool = True):
        """dL: fixed image gradient for the backward; or target: the step computes the
        squared-error loss against it (snp_mse_loss) and back-propagates its gradient
        (self.loss holds the loss after each replay).  reserve=False captures on the
        context's current reservation (same cameras, configuration and scene shape):
        several graphs over different scene and output buffers then share one set of
        workspace buffers, and must be replayed one after another on one stream."""
        self.r, self.ps, self.cams, self.cfg = renderer, ps, cams, cfg
        if reserve:
            renderer.reserve(ps, cams, cfg, max_keys)
        P = renderer.image_size(cams)
        self.image = torch.empty((P, 3), dtype=torch.float32, device=renderer.device)
        self.target = target
        self.loss = torch.zeros(1, dtype=torch.float32, device=renderer.device) if target is not None else None
        if target is not None:
            dL = torch.empty((P, 3), dtype=torch.float32, device=renderer.device)
        elif backward and dL is None:
            raise ValueError("GraphStep needs dL or target for the backward")
        self.dL = dL
        self.g_geom = torch.zeros_like(ps.geom) if backward else None
        self.g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device=ps.net.device) if backward else None
        self.backward = backward
        side = torch.cuda.Stream(renderer.device)
        side.wait_stream(torch.cuda.current_stream(renderer.device))
        with torch.cuda.stream(side):
            self._body()  # warm-up outside the capture (sets kernel attributes)
        torch.cuda.current_stream(renderer.device).wait_stream(side)
        torch.cuda.synchronize(renderer.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()
        self.token = renderer.token

    def _body(self):
        if self.backward:
            self.g_geom.zero_()
            self.g_net.zero_()
        self.r.forward(self.ps, self.cams, self.cfg, out=self.image)
        if self.target is not None:
            self.r.mse_loss(self.image, self.target, self.dL, self.loss)
        if self.backward:
            self.r.backward(self.ps, self.dL, self.g_geom, self.g_net)

    def replay(self):
        self.graph.replay()


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


# The differentiable render under its public name: images as a function of the
# packed geometry and network tensors (snp_render_forward / snp_render_backward).
SplatNetRender = _RenderFn


def render(renderer: Renderer, ps: PackedScene, cams, cfg: Optional[L.Config] = None) -> torch.Tensor:
    """Differentiable render: images [sum H*W, 3] (views concatenated, HWC) as a function of
    ps.geom and ps.net (set requires_grad on them to get gradients)."""
    return _RenderFn.apply(ps.geom, ps.net, renderer, ps, cams, cfg or L.make_config())
