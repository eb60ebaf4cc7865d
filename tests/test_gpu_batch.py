"""Batched multi-view rendering (rg_render_batch) through the C ABI.

Each image of a batch must equal, bit for bit, the single-view rg_render image
of the same scene and camera with the pixels-per-thread variant the batch's
autotuner chose (the kernels are deterministic), and sampled tiles of every
view must match the FP64 oracle with the tile shape the plan uses, under the
same tolerances as the single-view parity tests. Views mix resolutions and two
resident scenes; a second call with new poses exercises the in-place graph
update, and RG_FLAG_BATCH_CHECKED the re-sizing after an overflow.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2608_15785_gb300 import binding, synth
from tests._parity import check_view, sample_tiles

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_15785_gb300.build import build
    build()


SOURCES = [synth.tiny_scene(10_000, seed=0), synth.clustered_scene(60_000, seed=5)]


@pytest.fixture(scope="module")
def scenes():
    return [binding.Scene(sc) for sc in SOURCES]


SIZES = [(256, 256), (320, 200), (640, 360), (100, 37), (512, 288), (1280, 720)]


def _cams(k0, zfar_far=56.5):
    cams = []
    for v, (w, h) in enumerate(SIZES):
        if v % 2 == 0:
            c = synth.look_at_camera((0.3 * np.sin(k0 + v), -0.2, -3.0), w, h, zfar=4.8)
        else:
            c = synth.orbit_camera(k0 + 3 * v, w, h, zfar=zfar_far)
        cams.append(c)
    return cams


def _single(scene, cam, mode, ppt, tile):
    flags = 0
    if mode == "roofgs":
        flags = {1: binding.RG_FLAG_SINGLE_PIXEL, 2: 0, 4: binding.RG_FLAG_QUAD_PIXEL}[ppt]
    out = scene.render(cam, mode=mode, flags=flags, tile=tile)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode,path", [("roofgs", "auto"), ("roofgs", "fused"), ("roofgs", "lanes"),
                                       ("exact", "auto")])
def test_batch_equals_single_views(scenes, mode, path):
    """path: the autotuner's choice, or forced: the fused path (one front-end launch over every
    view's Gaussians, one persistent rasterizer over every view's tiles) or the lanes."""
    idx = [v % 2 for v in range(len(SIZES))]
    pf = {"auto": 0, "fused": binding.RG_FLAG_BATCH_FUSED, "lanes": binding.RG_FLAG_BATCH_LANES}[path]
    for call, k0 in enumerate((0, 7)):  # second call: new poses, same plan (graph update)
        cams = _cams(k0)
        outs = binding.render_batch(scenes, idx, cams, mode=mode, flags=pf)
        torch.cuda.synchronize()
        lanes, ppt, tw, th, fused = binding.batch_plan_info(scenes, idx, cams, mode=mode, flags=pf, with_path=True)
        assert lanes in (1, 2, 4) and ppt in ((1, 2, 4) if mode == "roofgs" else (2,))
        assert (tw, th) in ((16, 16), (32, 8), (8, 32))
        if path != "auto":
            assert fused == (path == "fused")
        if mode == "exact":
            assert not fused
        for v, cam in enumerate(cams):
            img = outs[v].cpu().numpy()
            ref = _single(scenes[idx[v]], cam, mode, ppt, (tw, th))
            assert np.array_equal(img, ref), (mode, call, v)
            # the oracle, on a few sampled tiles of every view (both calls)
            tiles = sample_tiles(cam, 6, seed=10 * call + v, tile=(tw, th))
            check_view(img.astype(np.float64), SOURCES[idx[v]], cam, mode, tile=(tw, th), tiles=tiles,
                       max_flagged=0.05, label="batch call %d view %d" % (call, v))
    for s in scenes:
        s.check()


def test_batch_checked_overflow_regrows(scenes):
    idx = [1, 1]
    far = [synth.orbit_camera(2, 640, 360, radius=20.0, zfar=80.0), synth.orbit_camera(5, 640, 360, radius=20.0,
                                                                                       zfar=80.0)]
    binding.render_batch(scenes, idx, far, mode="roofgs")  # plan sized for far views (few entries)
    near = [synth.orbit_camera(2, 640, 360, radius=2.2, zfar=80.0), synth.orbit_camera(5, 640, 360, radius=2.2,
                                                                                        zfar=80.0)]
    outs = binding.render_batch(scenes, idx, near, mode="roofgs", flags=binding.RG_FLAG_BATCH_CHECKED)
    torch.cuda.synchronize()
    lanes, ppt, tw, th = binding.batch_plan_info(scenes, idx, near, mode="roofgs")
    for v, cam in enumerate(near):
        assert np.array_equal(outs[v].cpu().numpy(), _single(scenes[1], cam, "roofgs", ppt, (tw, th)))
    scenes[1].check()


@pytest.mark.parametrize("tile", [(32, 8), (8, 32)])
def test_batch_with_a_fixed_tile_shape(scenes, tile):
    idx = [v % 2 for v in range(len(SIZES))]
    cams = _cams(3)
    outs = binding.render_batch(scenes, idx, cams, mode="roofgs", tile=tile)
    torch.cuda.synchronize()
    lanes, ppt, tw, th = binding.batch_plan_info(scenes, idx, cams, mode="roofgs", tile=tile)
    assert (tw, th) == tile
    for v, cam in enumerate(cams):
        assert np.array_equal(outs[v].cpu().numpy(), _single(scenes[idx[v]], cam, "roofgs", ppt, tile))


def test_fused_path_limits(scenes):
    """The fused path renders RoofGS mode and at most 32 views; beyond that the autotuned plan
    takes the lanes, and its images still equal the single-view renders."""
    cams = _cams(1)[:2]
    with pytest.raises(binding.RgError) as e:
        binding.render_batch(scenes, [0, 1], cams, mode="exact", flags=binding.RG_FLAG_BATCH_FUSED)
    assert e.value.status == 8
    many = [synth.look_at_camera((0.05 * v - 0.8, -0.2, -3.0), 64 + 4 * (v % 3), 48, zfar=4.8) for v in range(33)]
    idx = [v % 2 for v in range(33)]
    with pytest.raises(binding.RgError) as e:
        binding.render_batch(scenes, idx, many, mode="roofgs", flags=binding.RG_FLAG_BATCH_FUSED)
    assert e.value.status == 8
    outs = binding.render_batch(scenes, idx, many, mode="roofgs")
    torch.cuda.synchronize()
    lanes, ppt, tw, th, fused = binding.batch_plan_info(scenes, idx, many, mode="roofgs", with_path=True)
    assert not fused
    for v in (0, 7, 32):
        assert np.array_equal(outs[v].cpu().numpy(), _single(scenes[idx[v]], many[v], "roofgs", ppt, (tw, th)))


@pytest.mark.parametrize("path", ["fused", "lanes"])
def test_batch_with_an_empty_view(scenes, path):
    """A view that sees no Gaussian (camera turned away: every Gaussian behind it) renders the
    background in both paths, beside ordinary views, and the others are unaffected."""
    pf = binding.RG_FLAG_BATCH_FUSED if path == "fused" else binding.RG_FLAG_BATCH_LANES
    away = synth.look_at_camera((0.0, 0.0, -3.0), 96, 64, zfar=4.8, target=(0.0, 0.0, -6.0), bg=(0.2, 0.4, 0.6))
    cams = [_cams(2)[0], away, _cams(2)[3]]
    idx = [0, 0, 1]
    outs = binding.render_batch(scenes, idx, cams, mode="roofgs", flags=pf)
    torch.cuda.synchronize()
    lanes, ppt, tw, th = binding.batch_plan_info(scenes, idx, cams, mode="roofgs", flags=pf)
    assert np.allclose(outs[1].cpu().numpy(), np.array([0.2, 0.4, 0.6])[:, None, None])
    for v, cam in enumerate(cams):
        assert np.array_equal(outs[v].cpu().numpy(), _single(scenes[idx[v]], cam, "roofgs", ppt, (tw, th))), v
