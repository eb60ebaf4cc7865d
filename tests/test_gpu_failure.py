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


def test_server_request_reports_the_timeout():
    """A request whose frame runs out its bounded wait comes back from rg_poll as
    RG_ERR_TIMEOUT; its slot is freed and a server without the hook serves normally."""
    sc = synth.tiny_scene(10_000, seed=0)
    cam = synth.tiny_camera(256, 256)
    gs = binding.Scene(sc)
    ref = gs.render(cam)
    torch.cuda.synchronize()
    out = torch.empty((3, 256, 256), device="cuda")
    for flags, expect in ((binding.RG_FLAG_TEST_STALL_SORT, RG_ERR_TIMEOUT), (0, 0)):
        srv = binding.Server([gs], 256, 256, mode="roofgs", flags=flags, max_slots=2)
        for _ in range(2):  # the freed slot takes the next request
            t = srv.submit(cam, 0)
            deadline, status = time.time() + 60.0, None
            while status is None and time.time() < deadline:
                try:
                    if srv.poll(t, out):
                        status = 0
                except binding.RgError as e:
                    status = e.status
                time.sleep(0.01)
            assert status == expect
            if expect == 0:
                torch.cuda.synchronize()
                assert torch.equal(out, ref)
        srv.close()
