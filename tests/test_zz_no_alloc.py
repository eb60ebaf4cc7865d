"""Allocation-free sort entry point (rg_sort_pairs_noalloc), called through the C ABI.

Callers that must not allocate device memory (real-time render threads,
plugins whose host owns all device memory, code recorded into CUDA graphs)
sort their own (key, value) arrays with scratch from a static device array.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.

The reference is the existing entry point: rg_render sorts the same entries
inside its frame, and rg_inspect returns that sorted result. The input given
to the allocation-free sort is the front end's emission order (Gaussian by
Gaussian, tiles ascending), so a stable sort must reproduce rg_render's output
bit for bit (integer results: exact equality). Two calls in a row check that
the contents the first call leaves in the shared scratch do not leak into the
second.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

from paper_2608_15785_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 19


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_15785_gb300.build import build
    build()
    return binding.lib()


def _render_sorted(gs, cam):
    gs.render(cam, mode="roofgs")
    torch.cuda.synchronize()
    return gs.inspect(binding.RG_INSPECT_KEYS).view(np.uint32).copy(), gs.inspect(binding.RG_INSPECT_VALUES).copy()


def _noalloc_sort(lib, keys, vals, key_bits=32):
    dk = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.rg_sort_pairs_noalloc(C.c_void_p(dk.data_ptr()), C.c_void_p(dv.data_ptr()), keys.size, key_bits,
                                       C.c_void_p(err.data_ptr()), stream)
    assert status == 0, lib.rg_last_error()
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return dk.cpu().numpy().view(np.uint32), dv.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_render_twice(lib):
    sc, cams = synth.workload("tiny_256")
    gs = binding.Scene(sc)
    cam2 = synth.look_at_camera((0.6, -0.3, -2.7), 240, 200, zfar=4.6)
    for cam in (cams[0], cam2):  # two calls in a row with different contents
        ref_k, ref_v = _render_sorted(gs, cam)
        assert 0 < ref_k.size <= MAX_PAIRS
        order = np.lexsort((ref_k, ref_v))  # emission order: by Gaussian, then tile
        got_k, got_v = _noalloc_sort(lib, ref_k[order], ref_v[order])
        assert np.array_equal(got_k, ref_k)
        assert np.array_equal(got_v, ref_v)


def test_noalloc_sort_partial_key_width_and_limits(lib):
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 2 ** 32, size=100_003, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    got_k, got_v = _noalloc_sort(lib, keys, vals, key_bits=24)  # 3 passes: result copied back
    order = np.argsort(keys & 0xFFFFFF, kind="stable")
    assert np.array_equal(got_v, vals[order]) and np.array_equal(got_k, keys[order])
    empty_k, empty_v = _noalloc_sort(lib, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert empty_k.size == 0
    status = lib.rg_sort_pairs_noalloc(None, None, MAX_PAIRS + 1, 32, None, None)
    assert status == 1 and b"524288" in lib.rg_last_error()


@pytest.mark.parametrize("key_bits", [16, 8])
def test_noalloc_sort_at_the_size_limit(lib, key_bits):
    """Exactly 524,288 random pairs: every look-back status row and the whole alternate
    buffers are used (16 bits: two passes, the result ends in the caller's arrays; 8 bits:
    one pass, the result is copied back from the scratch array)."""
    rng = np.random.default_rng(key_bits)
    keys = rng.integers(0, 2 ** 32, size=MAX_PAIRS, dtype=np.uint64).astype(np.uint32)
    vals = rng.permutation(MAX_PAIRS).astype(np.uint32)
    got_k, got_v = _noalloc_sort(lib, keys, vals, key_bits=key_bits)
    order = np.argsort(keys & np.uint32((1 << key_bits) - 1), kind="stable")
    assert np.array_equal(got_v, vals[order]) and np.array_equal(got_k, keys[order])
