"""Failure path on the GPU without a fault: a bounded device wait is made to run out
(RG_FLAG_TEST_STALL_SORT: the first radix pass never processes its first tile, so the
next tile's look-back waits for counts nobody publishes). The kernels give up after their
bounded wait, finish with in-bounds writes, and the host reads RG_ERR_TIMEOUT; the scene
and the CUDA context keep working."""
from __future__ import annotations

import time

import pytest

from paper_2608_15785_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RG_ERR_TIMEOUT = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_15785_gb300.build import build
    build()


@pytest.mark.parametrize("mode", ["roofgs", "exact"])
def test_stalled_lookback_times_out_and_reports(mode):
    sc = synth.tiny_scene(10_000, seed=0)
    cam = synth.tiny_camera(256, 256)
    gs = binding.Scene(sc)
    ref = gs.render(cam, mode=mode)
    torch.cuda.synchronize()
    gs.check()
    # unchecked frame: the timeout is reported by the next check
    t0 = time.time()
    gs.render(cam, mode=mode, flags=binding.RG_FLAG_TEST_STALL_SORT)
    torch.cuda.synchronize()
    assert time.time() - t0 < 30.0
    with pytest.raises(binding.RgError) as e:
        gs.check()
    assert e.value.status == RG_ERR_TIMEOUT
    gs.check()  # the sticky flag was cleared by the check that reported it
    # checked frame: the call itself reports it
    with pytest.raises(binding.RgError) as e:
        gs.render(cam, mode=mode, flags=binding.RG_FLAG_TEST_STALL_SORT, stats=True)
    assert e.value.status == RG_ERR_TIMEOUT
    try:
        gs.check()
    except binding.RgError as e2:
        assert e2.status == RG_ERR_TIMEOUT
    # the scene and the context still render the same image
    again = gs.render(cam, mode=mode)
    torch.cuda.synchronize()
    gs.check()
    assert torch.equal(again, ref)
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0
