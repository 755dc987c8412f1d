"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/snp.h declares.

No compute call is made (no GPU needed)."""
import ctypes

import pytest

from paper_2510_08491_gb300 import _lib as L


def test_header_declares_the_boundary():
    syms = L.header_symbols()
    for s in ("snp_create", "snp_destroy", "snp_render_forward", "snp_render_backward", "snp_reserve",
              "snp_debug_keys", "snp_get_stats", "snp_last_error", "snp_get_net_layout",
              "snp_default_chunks"):
        assert s in syms


def test_library_exports_every_header_symbol():
    from paper_2510_08491_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for s in L.header_symbols():
        assert hasattr(lib, s), s


def test_net_layout_is_aligned_and_complete():
    offs, stride = L.net_layout(16, L.COLOR_MLP, 32)
    sizes = [48, 16, 16, 1, 8, 32 * 11, 32, 32 * 32, 32, 96, 3]
    assert offs[11] == -1
    offs = offs[:11]
    assert all(o % 8 == 0 for o in offs) and stride % 8 == 0
    spans = sorted(zip(offs, sizes))
    for (o1, s1), (o2, _) in zip(spans, spans[1:]):
        assert o1 + s1 <= o2
    assert spans[-1][0] + spans[-1][1] <= stride
    offs_c, stride_c = L.net_layout(8, L.COLOR_CONST, 0)
    assert offs_c[4:] == [-1] * 10 and stride_c == 24 + 8 + 8 + 8
    # spherical harmonics: the density fields, then sh [16][3]
    offs_s, stride_s = L.net_layout(8, L.COLOR_SH, 0)
    assert offs_s[4:11] == [-1] * 7 and offs_s[11] == 48 and stride_s == 48 + 48
    assert offs_s[12:] == [-1, -1]
    # time-conditioned: W_t [N_sigma] after everything, then the SH series [12][3]
    offs_d, stride_d = L.net_layout(8, L.COLOR_SH, 0, dynamic=True)
    assert offs_d[:12] == offs_s[:12] and offs_d[12] == 96 and offs_d[13] == 104 and stride_d == 144
    offs_dc, stride_dc = L.net_layout(8, L.COLOR_CONST, 0, dynamic=True)
    assert offs_dc[12] == 48 and offs_dc[13] == -1 and stride_dc == 56
    with pytest.raises(L.SnpError):
        L.net_layout(8, L.COLOR_MLP, 32, dynamic=True)


def test_argument_errors_are_reported_before_any_device_work():
    """Calls with a null context, a bad description or bad sizes fail with the
    documented status before they touch the CUDA runtime (so they run here too)."""
    from paper_2510_08491_gb300 import build
    build.build()
    lib = L.lib()
    bad = L.SNP_ERR_INVALID_ARG
    null = None
    assert lib.snp_reserve(null, null, null, 1, null, 0) == bad
    assert lib.snp_render_forward(null, null, null, null, 1, null, null, null, null) == bad
    assert lib.snp_render_backward(null, 1, null, null, null, null, null) == bad
    assert lib.snp_get_stats(null, 1, null, null) == bad
    assert lib.snp_debug_keys(null, 1, null, null, 0, null, null) == bad
    assert lib.snp_stage_times(null, null, null, 0) == bad
    assert lib.snp_autotune(null, null, null, null, 1, null, 0, null, null, null) == bad
    assert lib.snp_mse_loss(null, null, null, 0, null, null, null) == bad
    assert lib.snp_popctl_accumulate(null, null, null, null, null, null) == bad
    assert lib.snp_popctl_plan(null, null, null, null, null, null, null, null, null, null) == bad
    assert lib.snp_popctl_apply(null, null, null, null, null, null, null, null, null) == bad
    assert lib.snp_geom_reg(null, null, null, 1.0, null, null, null) == bad
    assert lib.snp_adam_step(null, null, null, null, null, null, null, null, null, null, null, null) == bad
    assert lib.snp_create(0, null) == bad
    lib.snp_destroy(null)
    assert lib.snp_last_error(null) == b"null context"

    # scene descriptions: the layout query runs the same checks as every call
    def desc(**kw):
        d = L.SceneDesc()
        d.n, d.n_sigma, d.color_mode, d.n_c, d.weight_dtype, d.omega0, d.dynamic = 10, 8, L.COLOR_CONST, 0, 0, 30.0, 0
        for k, v in kw.items():
            setattr(d, k, v)
        return d
    out = L.NetLayout()
    assert lib.snp_get_net_layout(ctypes.byref(desc()), ctypes.byref(out)) == L.SNP_OK
    assert lib.snp_get_net_layout(null, ctypes.byref(out)) == bad
    for kw in ({"n": -1}, {"n": (1 << 28) + 1}, {"n_sigma": 0}, {"n_sigma": 65}, {"color_mode": 7},
               {"weight_dtype": 5}, {"dynamic": 2}):
        assert lib.snp_get_net_layout(ctypes.byref(desc(**kw)), ctypes.byref(out)) == bad, kw
    for kw in ({"color_mode": L.COLOR_MLP, "n_c": 48}, {"color_mode": L.COLOR_MLP, "n_c": 32, "dynamic": 1}):
        assert lib.snp_get_net_layout(ctypes.byref(desc(**kw)), ctypes.byref(out)) == L.SNP_ERR_UNSUPPORTED, kw

    # the allocation-free sort validates sizes before it looks for a device
    raw = ctypes.CDLL(build.LIB)
    f = raw.snp_sort_pairs_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    assert f(null, null, -1, 32, null) == bad
    assert f(null, null, 4, 0, null) == bad
    assert f(null, null, 4, 65, null) == bad
    assert f(null, null, (1 << 20) + 1, 32, null) == L.SNP_ERR_CAPACITY
    assert f(null, null, 4, 32, null) == bad
    # misaligned key (8-byte) or value (4-byte) pointers are refused before the device is touched
    assert f(4100, 8192, 4, 32, null) == bad
    assert f(8192, 4098, 4, 32, null) == bad


def test_default_chunks_follow_the_shared_memory_budgets():
    """snp_default_chunks is host-only.  At N_sigma = 16, N_c = 32 both passes stage 5
    entries (71.5 KB of the forward's three-CTA budget of 72 KB, 105 KB of the
    backward's two-CTA budget of 108 KB).  At N_sigma = 32, N_c = 64 the
    tensor-memory backward stages 4: the most its operand tiles can take at the
    chunk's end (4 x 16 KB), and 202 KB of shared memory.  Without a colour network
    the 16-pixel backward's masks allow 32 entries, and the budget gives 15 at
    N_sigma = 8 (106 KB), 14 time-conditioned (102 KB); 32-pixel tiles stay at
    8 or fewer.  Bad arguments are refused."""
    assert L.default_chunks(16, L.COLOR_MLP, 32) == (5, 5)
    f64, b64 = L.default_chunks(32, L.COLOR_MLP, 64)
    assert b64 == 4 and 1 <= f64 <= 32
    assert L.default_chunks(8, L.COLOR_SH, 0) == (32, 15)
    assert L.default_chunks(8, L.COLOR_SH, 0, dynamic=True) == (32, 14)
    f32t, b32t = L.default_chunks(8, L.COLOR_SH, 0, tile_size=32)
    assert 1 <= f32t <= 32 and 1 <= b32t <= 8
    assert L.default_chunks(16, L.COLOR_MLP, 32, tile_size=0) == (5, 5)
    lib = L.lib()
    d = L.SceneDesc(10, 16, L.COLOR_MLP, 32, 0, 30.0, 0)
    f, b = ctypes.c_int32(), ctypes.c_int32()
    assert lib.snp_default_chunks(None, 16, ctypes.byref(f), ctypes.byref(b)) == L.SNP_ERR_INVALID_ARG
    assert lib.snp_default_chunks(ctypes.byref(d), 16, None, ctypes.byref(b)) == L.SNP_ERR_INVALID_ARG
    assert lib.snp_default_chunks(ctypes.byref(d), 12, ctypes.byref(f), ctypes.byref(b)) == L.SNP_ERR_UNSUPPORTED
