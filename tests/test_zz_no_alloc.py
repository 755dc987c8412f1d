"""The allocation-free sort entry point (snp_sort_pairs_noalloc) through the C ABI.

Callers that cannot allocate device memory while they run (an application
whose memory pool owns the device, a plugin handed a fixed arena, a loop that
cannot take cudaMalloc's implicit synchronisation) sort with scratch that lives
in a static device array of the library.  This checks, on two calls
in a row with different inputs, that it orders the tile keys exactly as the
sort inside snp_render_forward does and as the oracle's stable sort does, that
key bits above the sorted width do not change the order, that the device's free
memory does not move across calls, and that it rejects sizes above its limit.
Kept in a file of its own that is collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    from paper_2510_08491_gb300 import _lib as L
    f = L.lib().snp_sort_pairs_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]
    f.restype = C.c_int32
    return f


def _tile_bits(tiles):
    b = 1
    while (1 << b) < tiles:
        b += 1
    return b


def test_noalloc_sort_matches_render_sort(oracle_lib):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300 import build
    from paper_2510_08491_gb300.render import Renderer, pack_scene
    build.build()
    O = oracle_lib
    sort = _noalloc_fn()
    r = Renderer(0)
    st = torch.cuda.current_stream().cuda_stream
    cases = [(synth.make_scene(3000, seed=21, center_half=3.0, n_sigma=8), synth.ring_cameras(2, 8.0, 320, 200)),
             (synth.make_scene(8000, seed=22, center_half=2.0, n_sigma=8), synth.ring_cameras(3, 6.0, 256, 256))]
    for sc, cams in cases:
        # the existing entry point: render, then read its sorted keys back
        r.forward(pack_scene(sc), cams, L.make_config())
        ref_k, ref_v = r.debug_keys()
        # the oracle's own stable sort of the same keys
        tl = O.tile_keys(sc, cams, 16)
        # the same keys in emission order (key specification of the oracle) sorted without allocating
        k, v, _, vto = O.emission_keys(sc, cams, 16)
        assert len(k) == len(ref_k) and 0 < len(k) <= (1 << 20)
        dk = torch.from_numpy(k.view(np.int64)).cuda()
        dv = torch.from_numpy(v.view(np.int32)).cuda()
        bits = 32 + _tile_bits(int(vto[-1]))
        assert sort(dk.data_ptr(), dv.data_ptr(), len(k), bits, st) == L.SNP_OK
        torch.cuda.synchronize()
        got_k, got_v = dk.cpu().numpy().view(np.uint64), dv.cpu().numpy().view(np.uint32)
        assert np.array_equal(got_k, ref_k) and np.array_equal(got_v, ref_v)
        assert np.array_equal(got_k, tl.keys) and np.array_equal(got_v, tl.vals)


def test_noalloc_sort_ignores_bits_above_key_bits_and_allocates_nothing():
    from paper_2510_08491_gb300 import _lib as L
    sort = _noalloc_fn()
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(7)
    n, bits = 300_000, 33
    low = rng.integers(0, 1 << bits, size=n, dtype=np.uint64) & np.uint64(0xFFF00000F)  # many equal keys
    junk = rng.integers(0, 1 << (64 - bits), size=n, dtype=np.uint64) << np.uint64(bits)
    keys = low | junk
    vals = np.arange(n, dtype=np.uint32)
    order = np.argsort(low, kind="stable")
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    assert sort(dk.data_ptr(), dv.data_ptr(), n, bits, st) == L.SNP_OK  # warm-up: kernels loaded, address looked up
    torch.cuda.synchronize()
    assert np.array_equal(dv.cpu().numpy().view(np.uint32), vals[order])
    assert np.array_equal(dk.cpu().numpy().view(np.uint64), keys[order])
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):  # two more calls in a row on fresh inputs
        dk.copy_(torch.from_numpy(keys.view(np.int64)))
        dv.copy_(torch.from_numpy(vals.view(np.int32)))
        assert sort(dk.data_ptr(), dv.data_ptr(), n, bits, st) == L.SNP_OK
        torch.cuda.synchronize()
        assert np.array_equal(dv.cpu().numpy().view(np.uint32), vals[order])
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0


def test_noalloc_sort_rejects_oversize():
    from paper_2510_08491_gb300 import _lib as L
    sort = _noalloc_fn()
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert sort(buf.data_ptr(), buf.data_ptr(), (1 << 20) + 1, 40, st) == L.SNP_ERR_CAPACITY
    assert sort(buf.data_ptr(), buf.data_ptr(), 4, 0, st) == L.SNP_ERR_INVALID_ARG
