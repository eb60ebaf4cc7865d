"""GPU parity of the renderer (through the C ABI) against the CPU oracle.

Bars (tolerances in tests/_parity.py):
  * bit-exact: compact attributes (FP16 geometry, log o, INT8 SH codes and
    scales), the bit-level exponential, sorted keys/values and tile ranges;
  * exact mode: |GPU - FP64 oracle| <= 2e-4 per channel on every pixel, except
    the colour jump of a skip/stop decision that lies within single-precision
    rounding of its threshold (diag[1], diag[2]); the share of pixels that
    carry such a flag is asserted to be small;
  * RoofGS mode: within eps_max = 0.0312 (the measured bound of Eq. (24)) of
    the oracle with exact exp, within 2e-4 + FP16 colour rounding (+ the
    oracle's FP32 estimate) of the oracle that evaluates Eq. (24) in FP32, and
    >= 46.4 dB PSNR against exact mode (0.05 dB against a 27 dB reference
    error).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2608_15785_gb300 import binding, synth
from tests._helpers import single_scene, small_random_scene
from tests._parity import HALF_COLOUR, ROOFGS_FLAGGED, TOL, check, check_view, sample_tiles

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_15785_gb300.build import build
    build()


def gpu_scene(sc, per_gauss=False):
    return binding.Scene(sc, sh_scale_mode=binding.RG_SH_SCALE_BAND_GAUSS if per_gauss else binding.RG_SH_SCALE_BAND)


def render(gs, cam, mode, flags=0, stats=False, tile=(16, 16)):
    out = gs.render(cam, mode=mode, flags=flags, stats=stats, tile=tile)
    torch.cuda.synchronize()
    if stats:
        return out[0].cpu().numpy().astype(np.float64), out[1]
    return out.cpu().numpy().astype(np.float64)


def assert_close(img, ref, diag, base, max_flagged=0.01, label="", fp32=False):
    """Every value within base + the flip allowance (+ the FP32 estimate for the RoofGS
    checks against the FP32 fast-exp oracle)."""
    return check(img, ref, diag, base, fp32=fp32, max_flagged=max_flagged, label=label)


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else -10 * math.log10(mse)


# ---------------------------------------------------------------------------
# bit-exact pieces
# ---------------------------------------------------------------------------

def test_fast_exp_bit_exact_against_fp32_formula():
    lo = np.float32(-oracle.LN255)
    a = np.uint32(np.float32(-0.0).view(np.uint32))
    b = np.uint32(lo.view(np.uint32))
    # every 7th FP32 value of [-ln 255, 0] plus the end points
    P = np.concatenate([np.arange(a, b + 1, 7, dtype=np.uint32).view(np.float32), [lo, np.float32(0)]])
    got = binding.eval_fast_exp(torch.from_numpy(P).cuda()).cpu().numpy()
    ref = oracle.fast_exp_many(P.astype(np.float64), oracle.EXP_FAST32).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("per_gauss", [False, True])
def test_compact_attributes_bit_exact(per_gauss):
    sc = synth.tiny_scene(20_000, seed=5)
    gs = gpu_scene(sc, per_gauss)
    comp = oracle.compact(sc, per_gauss)
    codes = gs.inspect(binding.RG_INSPECT_SH_CODES).reshape(sc.n, 16, 3)
    assert np.array_equal(codes, comp.codes)
    assert np.array_equal(gs.inspect(binding.RG_INSPECT_SH_SCALES).reshape(4, 3).view(np.uint32),
                          comp.band_scale.view(np.uint32))
    g16 = gs.inspect(binding.RG_INSPECT_GEOM16).reshape(sc.n, 8)
    assert np.array_equal(g16[:, 0:4], sc.quats.astype(np.float16).view(np.uint16))
    assert np.array_equal(g16[:, 4:7], sc.scales.astype(np.float16).view(np.uint16))
    assert np.array_equal(g16[:, 7], comp.gauss_scale.astype(np.float16).view(np.uint16))
    assert np.array_equal(gs.inspect(binding.RG_INSPECT_LOG_OPACITY).view(np.uint32), comp.log_opac.view(np.uint32))


def _keys_equal(gs, sc, cam, mode, comp=None, tile=(16, 16)):
    k, v, ranges, _ = oracle.keys(sc, cam, mode, comp=comp, tile=tile)
    gk = gs.inspect(binding.RG_INSPECT_KEYS)
    gk = gk.view(np.uint64) if mode == oracle.EXACT else gk.view(np.uint32).astype(np.uint64)
    gv = gs.inspect(binding.RG_INSPECT_VALUES)
    gr = gs.inspect(binding.RG_INSPECT_RANGES).reshape(-1, 2)
    assert gk.size == k.size, (gk.size, k.size)
    assert np.array_equal(gk, k)
    assert np.array_equal(gv, v)
    assert np.array_equal(gr, ranges)
    return k.size


@pytest.mark.parametrize("mode", [oracle.EXACT, oracle.ROOFGS])
def test_keys_values_ranges_bit_exact_tiny(mode):
    sc, cams = synth.workload("tiny_256")
    gs = gpu_scene(sc)
    comp = oracle.compact(sc) if mode == oracle.ROOFGS else None
    _, st = render(gs, cams[0], mode, stats=True)
    n = _keys_equal(gs, sc, cams[0], mode, comp)
    assert st["n_entries"] == n
    # RoofGS: Gaussians depth-ordered first, then one 8-bit pass over the 8 tile bits;
    # exact: 32 depth bits + 8 tile bits -> 5 digits
    assert st["sort_passes"] == (1 if mode == oracle.ROOFGS else 5)
    if mode == oracle.ROOFGS:  # the paper's 4-pass full-key sort gives the same entries
        _, st4 = render(gs, cams[0], "roofgs", flags=binding.RG_FLAG_SORT_FULL_KEY, stats=True)
        assert st4["sort_passes"] == 4
        _keys_equal(gs, sc, cams[0], mode, comp)


# ---------------------------------------------------------------------------
# images
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny():
    sc, cams = synth.workload("tiny_256")
    return sc, cams[0], gpu_scene(sc), oracle.compact(sc)


def test_exact_mode_matches_oracle_tiny(tiny):
    sc, cam, gs, _ = tiny
    img = render(gs, cam, "exact")
    ref, diag, _ = oracle.render(sc, cam, oracle.EXACT)
    err, flagged = assert_close(img, ref, diag, TOL, label="exact tiny")
    print("exact tiny: max err %.3g, flagged %.4f" % (err, flagged))


def test_roofgs_mode_within_fast_exp_bound_tiny(tiny):
    sc, cam, gs, comp = tiny
    img = render(gs, cam, "roofgs")
    ref, diag, _ = oracle.render(sc, cam, oracle.ROOFGS, comp=comp)
    assert_close(img, ref, diag, oracle.EPS_MAX + TOL + HALF_COLOUR, max_flagged=ROOFGS_FLAGGED,
                 label="roofgs vs exact exp")
    ref32, diag32, _ = oracle.render(sc, cam, oracle.ROOFGS, comp=comp, exp_kind=oracle.EXP_FAST32)
    err, flagged = assert_close(img, ref32, diag32, TOL + HALF_COLOUR, max_flagged=ROOFGS_FLAGGED, fp32=True,
                                label="roofgs vs fp32 fast exp")
    print("roofgs tiny vs fast-exp oracle: max err %.3g, flagged %.4f" % (err, flagged))


@pytest.mark.parametrize("flags", [binding.RG_FLAG_EXACT_EXP, binding.RG_FLAG_SINGLE_PIXEL,
                                   binding.RG_FLAG_EXACT_EXP | binding.RG_FLAG_SINGLE_PIXEL,
                                   binding.RG_FLAG_QUAD_PIXEL, binding.RG_FLAG_EXACT_EXP | binding.RG_FLAG_QUAD_PIXEL,
                                   binding.RG_FLAG_SORT_FULL_KEY])
def test_roofgs_ingredient_toggles(tiny, flags):
    sc, cam, gs, comp = tiny
    img = render(gs, cam, "roofgs", flags=flags)
    kind = oracle.EXP_EXACT if flags & binding.RG_FLAG_EXACT_EXP else oracle.EXP_FAST32
    ref, diag, _ = oracle.render(sc, cam, oracle.ROOFGS, comp=comp, exp_kind=kind)
    assert_close(img, ref, diag, TOL + HALF_COLOUR, max_flagged=ROOFGS_FLAGGED, fp32=True, label="flags %d" % flags)


@pytest.mark.parametrize("flags", [0, binding.RG_FLAG_SINGLE_PIXEL, binding.RG_FLAG_QUAD_PIXEL, binding.RG_FLAG_EXACT_EXP])
def test_timed_launch_equals_counting_launch(flags):
    """The counting launch of a stats call and the launch timed by the benchmark are
    separate kernel variants: both must give the same bits, on close, far,
    thin-Gaussian and ragged views."""
    needles = synth.tiny_scene(4000, seed=7)
    rng = np.random.default_rng(7)
    needles.scales = (needles.scales * np.where(rng.random((4000, 3)) < 0.5, 0.02, 6.0)).astype(np.float32)
    cases = [(synth.tiny_scene(10_000, seed=0), [synth.tiny_camera(256, 256), synth.tiny_camera(100, 37)]),
             (needles, [synth.tiny_camera(320, 200), synth.tiny_camera(97, 131)]),
             (synth.clustered_scene(200_000, seed=3), [synth.orbit_camera(k, 1280, 720, radius=r)
                                                       for k, r in ((0, 4.0), (5, 1.6), (9, 12.0))])]
    for sc, cams in cases:
        gs = gpu_scene(sc)
        for cam in cams:
            a, _ = render(gs, cam, "roofgs", flags=flags, stats=True)
            b = render(gs, cam, "roofgs", flags=flags)
            assert np.array_equal(a, b), (cam.width, cam.height)
            assert a.std() > 0


def test_outputs_are_finite_and_in_range():
    """NaN/Inf scan of the images of every mode and ingredient, on close, far and thin views."""
    sc = synth.clustered_scene(200_000, seed=3)
    gs = gpu_scene(sc)
    cams = [synth.orbit_camera(k, 640, 360, radius=r) for k, r in ((0, 4.0), (5, 1.2), (9, 30.0))]
    flag_sets = [0, binding.RG_FLAG_EXACT_EXP, binding.RG_FLAG_SINGLE_PIXEL, binding.RG_FLAG_QUAD_PIXEL,
                 binding.RG_FLAG_SORT_FULL_KEY]
    for cam in cams:
        for mode in ("exact", "roofgs"):
            for fl in (flag_sets if mode == "roofgs" else [0]):
                img = render(gs, cam, mode, flags=fl)
                assert np.isfinite(img).all(), (mode, fl)
                # colours in [0, 1] blended with weights summing to 1 - T, plus T bg
                assert img.min() >= -1e-6 and img.max() <= 1.0 + 1e-5, (mode, fl, img.min(), img.max())
    gs.check()


def test_roofgs_psnr_against_exact_tiny(tiny):
    sc, cam, gs, _ = tiny
    a = render(gs, cam, "exact")
    b = render(gs, cam, "roofgs")
    assert psnr(a, b) >= 46.4


def test_deterministic_and_per_gaussian_sh_scale(tiny):
    sc, cam, gs, _ = tiny
    a = render(gs, cam, "roofgs")
    b = render(gs, cam, "roofgs")
    assert np.array_equal(a, b)
    e1 = render(gs, cam, "exact")
    e2 = render(gs, cam, "exact")
    assert np.array_equal(e1, e2)
    gp = gpu_scene(sc, per_gauss=True)
    comp = oracle.compact(sc, True)
    img = render(gp, cam, "roofgs")
    ref, diag, _ = oracle.render(sc, cam, oracle.ROOFGS, comp=comp, exp_kind=oracle.EXP_FAST32)
    assert_close(img, ref, diag, TOL + HALF_COLOUR, max_flagged=ROOFGS_FLAGGED, fp32=True,
                 label="per-gaussian sh scale")


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["exact", "roofgs"])
@pytest.mark.parametrize("wh", [(100, 37), (16, 16), (1, 1), (33, 250)])
def test_ragged_image_sizes(mode, wh):
    sc = small_random_scene(300, seed=21)
    cam = synth.tiny_camera(wh[0], wh[1], bg=(0.1, 0.2, 0.3))
    gs = gpu_scene(sc)
    om = oracle.EXACT if mode == "exact" else oracle.ROOFGS
    comp = oracle.compact(sc) if mode == "roofgs" else None
    img, st = render(gs, cam, mode, stats=True)
    ref, diag, _ = oracle.render(sc, cam, om, comp=comp, exp_kind=oracle.EXP_FAST32)
    assert_close(img, ref, diag, TOL + (HALF_COLOUR if mode == "roofgs" else 0),
                 max_flagged=0.05 if mode == "exact" else ROOFGS_FLAGGED, fp32=mode == "roofgs", label=str(wh))
    _keys_equal(gs, sc, cam, om, comp)


@pytest.mark.parametrize("mode", ["exact", "roofgs"])
def test_empty_and_fully_culled_scenes(mode):
    cam = synth.tiny_camera(64, 48, bg=(0.25, 0.5, 0.75))
    empty = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                        np.zeros(0, np.float32), np.zeros((0, 16, 3), np.float32))
    img, st = render(gpu_scene(empty), cam, mode, stats=True)
    assert st["n_entries"] == 0
    assert np.allclose(img, np.array([0.25, 0.5, 0.75])[:, None, None])
    behind = small_random_scene(50, seed=3)
    behind.means[:, 2] = -10.0  # behind the camera (z < znear)
    img, st = render(gpu_scene(behind), cam, mode, stats=True)
    assert st["n_entries"] == 0 and st["n_front"] == 0
    assert np.allclose(img, np.array([0.25, 0.5, 0.75])[:, None, None])


def test_degenerate_gaussians_are_culled_consistently():
    sc = small_random_scene(64, seed=8)
    sc.quats[:5] = 0.0            # zero quaternion: culled on both sides
    sc.opacities[5:10] = 1e-3     # below 1/255: culled in RoofGS mode
    sc.opacities[10:12] = 0.0
    sc.scales[12:15] = 0.0        # zero scale: only the 0.3 dilation remains
    cam = synth.tiny_camera(64, 64)
    gs = gpu_scene(sc)
    for mode, om in (("exact", oracle.EXACT), ("roofgs", oracle.ROOFGS)):
        comp = oracle.compact(sc) if mode == "roofgs" else None
        img = render(gs, cam, mode)
        ref, diag, _ = oracle.render(sc, cam, om, comp=comp, exp_kind=oracle.EXP_FAST32)
        assert_close(img, ref, diag, TOL + HALF_COLOUR, max_flagged=0.05 if mode == "exact" else ROOFGS_FLAGGED,
                     fp32=mode == "roofgs", label=mode)
        _keys_equal(gs, sc, cam, om, comp)


def test_invalid_inputs_are_rejected():
    sc = small_random_scene(10, seed=1)
    bad = sc.subset(np.arange(10))
    bad.means[3, 1] = np.nan
    with pytest.raises(binding.RgError) as e:
        gpu_scene(bad)
    assert e.value.status == 1
    bad = sc.subset(np.arange(10))
    bad.opacities[2] = 1.5
    with pytest.raises(binding.RgError):
        gpu_scene(bad)
    gs = gpu_scene(sc)
    cam = synth.tiny_camera(32, 32)
    cam.zfar = cam.znear
    with pytest.raises(binding.RgError):
        gs.render(cam)
    cam = synth.tiny_camera(32, 32)
    c = binding.camera_struct(cam)
    o = binding.RgOpts(binding.RG_MODE_ROOFGS, 0, 8, 8)
    out = torch.empty((3, 32, 32), device="cuda")
    import ctypes as C
    assert binding.lib().rg_render(gs.handle, C.byref(c), C.byref(o), C.c_void_p(out.data_ptr()), None,
                                   C.c_void_p(0)) == 8  # other tile shapes are not built


def test_capacity_overflow_regrows_and_is_reported():
    sc, cams = synth.workload("tiny_256")
    cam = cams[0]
    gs = gpu_scene(sc)
    ref = render(gs, cam, "roofgs")
    small = gpu_scene(sc)
    small.reserve(1000)  # far below the ~27k entries of this frame
    # asynchronous render: image incomplete, overflow recorded
    small.render(cam, flags=binding.RG_FLAG_ORDERED_FRONT_END)
    torch.cuda.synchronize()
    # the sort covers the entries that fit, i.e. the first ones the fused front end emitted
    # (Gaussians in (depth code, index) order, each one's tiles ascending): its digit
    # counts are taken from the stored keys, not from the front end's count of all
    gk = small.inspect(binding.RG_INSPECT_KEYS).view(np.uint32).astype(np.uint64)
    gv = small.inspect(binding.RG_INSPECT_VALUES)
    k, v, _, _ = oracle.keys(sc, cam, oracle.ROOFGS, comp=oracle.compact(sc))
    b_d = np.uint64(oracle.layout(cam)["b_d"])
    assert 0 < gk.size < k.size
    emitted = np.lexsort((k >> b_d, v, k & ((np.uint64(1) << b_d) - np.uint64(1))))[: gk.size]
    expect = emitted[np.lexsort((v[emitted], k[emitted]))]
    assert np.array_equal(gk, k[expect]) and np.array_equal(gv, v[expect])
    with pytest.raises(binding.RgError) as e:
        small.check()
    assert e.value.status == 4
    small.check()  # flags were cleared
    img, st = render(small, cam, "roofgs", stats=True)
    assert st["regrown"] == 1 and st["capacity"] >= st["n_entries"]
    assert np.array_equal(img, ref)
    small.check()


def test_exact_capacity_overflow_recounts_digits():
    """Exact mode with too small a workspace: the entries that fit are the first ones the
    duplicate kernel emitted (Gaussian by Gaussian, tiles ascending), and their sort must
    not use the duplicate kernel's digit counts (which cover every entry): the clipped
    sort equals the oracle's first entries, sorted. A checked render then regrows."""
    sc, cams = synth.workload("tiny_256")
    cam = cams[0]
    ref = render(gpu_scene(sc), cam, "exact")
    small = gpu_scene(sc)
    small.reserve(3000)
    small.render(cam, mode="exact")
    torch.cuda.synchronize()
    gk = small.inspect(binding.RG_INSPECT_KEYS).view(np.uint64)
    gv = small.inspect(binding.RG_INSPECT_VALUES)
    k, v, _, _ = oracle.keys(sc, cam, oracle.EXACT)
    assert 0 < gk.size < k.size
    emitted = np.lexsort((k, v))[: gk.size]
    expect = emitted[np.lexsort((v[emitted], k[emitted]))]
    assert np.array_equal(gk, k[expect]) and np.array_equal(gv, v[expect])
    with pytest.raises(binding.RgError) as e:
        small.check()
    assert e.value.status == 4
    img, st = render(small, cam, "exact", stats=True)
    assert st["regrown"] == 1 and np.array_equal(img, ref)
    small.check()


@pytest.mark.parametrize("name", ["tiny_256", "clustered_1080p", "clustered_4k"])
def test_tile_counting_sort_matches_the_radix_passes(name):
    """RG_FLAG_TILE_COUNTING_SORT groups the depth-ordered entries by tile with one stable
    counting sort: keys, values and ranges bit-exact against the oracle, the image bit-identical
    to the radix path's (2 and 4 pixels per thread)."""
    sc, cams = synth.workload(name)
    cam = cams[0] if name != "clustered_4k" else cams[7]
    per_gauss = name == "clustered_4k"
    gs = gpu_scene(sc, per_gauss)
    comp = oracle.compact(sc, per_gauss)
    for ppt in (0, binding.RG_FLAG_QUAD_PIXEL):
        ref, st = render(gs, cam, "roofgs", flags=ppt, stats=True)
        img, st2 = render(gs, cam, "roofgs", flags=ppt | binding.RG_FLAG_TILE_COUNTING_SORT, stats=True)
        assert st2["n_entries"] == st["n_entries"]
        assert np.array_equal(img, ref)
        assert st2["n_entries"] == _keys_equal(gs, sc, cam, oracle.ROOFGS, comp)
        # the timed (unchecked) launch gives the same image
        assert np.array_equal(render(gs, cam, "roofgs", flags=ppt | binding.RG_FLAG_TILE_COUNTING_SORT), ref)
    gs.check()


def test_tile_counting_sort_limits_and_overflow():
    """The counting sort needs the depth pre-sort and 16-bit tile ids (RG_ERR_UNSUPPORTED
    otherwise); an overflowed frame sorts exactly its first emitted entries."""
    sc, cams = synth.workload("tiny_256")
    cam = cams[0]
    gs = gpu_scene(sc)
    with pytest.raises(binding.RgError) as e:
        gs.render(cam, flags=binding.RG_FLAG_TILE_COUNTING_SORT | binding.RG_FLAG_SORT_FULL_KEY)
    assert e.value.status == 8
    with pytest.raises(binding.RgError) as e:  # 7680 x 4320: 17 tile bits
        gs.render(synth.orbit_camera(0, 7680, 4320), flags=binding.RG_FLAG_TILE_COUNTING_SORT)
    assert e.value.status == 8
    small = gpu_scene(sc)
    small.reserve(1000)
    small.render(cam, flags=binding.RG_FLAG_TILE_COUNTING_SORT)
    torch.cuda.synchronize()
    gk = small.inspect(binding.RG_INSPECT_KEYS).view(np.uint32).astype(np.uint64)
    gv = small.inspect(binding.RG_INSPECT_VALUES)
    k, v, _, _ = oracle.keys(sc, cam, oracle.ROOFGS, comp=oracle.compact(sc))
    b_d = np.uint64(oracle.layout(cam)["b_d"])
    assert 0 < gk.size < k.size
    emitted = np.lexsort((k >> b_d, v, k & ((np.uint64(1) << b_d) - np.uint64(1))))[: gk.size]
    expect = emitted[np.lexsort((v[emitted], k[emitted]))]
    assert np.array_equal(gk, k[expect]) and np.array_equal(gv, v[expect])
    with pytest.raises(binding.RgError):
        small.check()
    img, st = render(small, cam, "roofgs", flags=binding.RG_FLAG_TILE_COUNTING_SORT, stats=True)
    assert st["regrown"] == 1 and np.array_equal(img, render(gs, cam, "roofgs"))
    small.check()


def test_stage_times_and_counters(tiny):
    sc, cam, gs, _ = tiny
    for _ in range(3):
        gs.render(cam, flags=binding.RG_FLAG_STAGE_EVENTS)
    ms, frames = gs.stage_times()
    assert frames == 3 and all(m >= 0 for m in ms) and ms[6] > 0
    assert abs(sum(ms[:6]) - ms[6]) < 0.05 * ms[6] + 1e-3
    _, st = render(gs, cam, "roofgs", stats=True)
    assert 0 < st["n_visible"] <= st["n_front"] <= sc.n
    assert st["n_blends"] <= st["n_pairs"]
    assert st["n_pairs"] > 0


# ---------------------------------------------------------------------------
# full-size workloads: bit-exact keys, sampled tiles against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,per_gauss", [("clustered_1080p", False), ("clustered_4k", True)])
def test_full_size_parity(name, per_gauss):
    sc, cams = synth.workload(name)
    cam = cams[0] if name == "clustered_1080p" else cams[7]
    gs = gpu_scene(sc, per_gauss)
    comp = oracle.compact(sc, per_gauss)
    tiles = sample_tiles(cam, 48, seed=1)
    for mode, om in (("exact", oracle.EXACT), ("roofgs", oracle.ROOFGS)):
        img, st = render(gs, cam, mode, stats=True)
        assert st["n_entries"] == _keys_equal(gs, sc, cam, om, comp if mode == "roofgs" else None)
        # RoofGS: the default two pixels per thread, and the four of the benchmark's timed frames
        variants = [("", img)] if mode == "exact" else [
            (" ppt2", img), (" ppt4", render(gs, cam, mode, flags=binding.RG_FLAG_QUAD_PIXEL))]
        for label, im in variants:
            check_view(im, sc, cam, mode, tiles=tiles, comp=comp, max_flagged=0.01, label=name + label)
    a = render(gs, cam, "exact")
    b = render(gs, cam, "roofgs")
    assert psnr(a, b) >= 46.4, psnr(a, b)
    b4 = render(gs, cam, "roofgs", flags=binding.RG_FLAG_QUAD_PIXEL)
    assert psnr(a, b4) >= 46.4, psnr(a, b4)


def test_8k_three_tile_bit_passes_and_seven_exact_passes():
    """7680x4320: 129,600 tiles, so b_t = 17 and b_d = 15 (Eq. (9)); the RoofGS tile-bit sort
    takes 3 passes and the exact 64-bit sort 7. Keys bit-exact, sampled tiles against the oracle."""
    cam = synth.orbit_camera(4, 7680, 4320)
    lay = oracle.layout(cam)
    assert (lay["b_t"], lay["b_d"]) == (17, 15)
    tiles = sample_tiles(cam, 32, seed=3)
    for mode, om, n in (("roofgs", oracle.ROOFGS, 300_000), ("exact", oracle.EXACT, 100_000)):
        sc = synth.clustered_scene(n, seed=6)
        gs = gpu_scene(sc, per_gauss=True)
        comp = oracle.compact(sc, True) if mode == "roofgs" else None
        img, st = render(gs, cam, mode, stats=True)
        assert st["sort_passes"] == (3 if mode == "roofgs" else 7)
        assert st["n_entries"] == _keys_equal(gs, sc, cam, om, comp)
        images = [img] if mode == "exact" else [img, render(gs, cam, mode, flags=binding.RG_FLAG_QUAD_PIXEL)]
        for im in images:
            check_view(im, sc, cam, mode, tiles=tiles, comp=comp, max_flagged=0.01, label="8k")
        gs.check()


@pytest.mark.parametrize("tile", [(32, 8), (8, 32)])
@pytest.mark.parametrize("mode", ["exact", "roofgs"])
def test_tile_shapes_bit_exact_keys_and_images(tile, mode):
    """32x8 and 8x32 tiles: keys, values and ranges bit-exact against the oracle's binning
    with the same tile shape, images within the tolerances, on square, ragged and 1080p views."""
    om = oracle.EXACT if mode == "exact" else oracle.ROOFGS
    sc, cams = synth.workload("tiny_256")
    cases = [(sc, cams[0], None), (sc, synth.tiny_camera(100, 37), None)]
    big, bcams = synth.workload("clustered_1080p")
    cases.append((big, bcams[0], sample_tiles(bcams[0], 48, seed=5, tile=tile)))
    for scene, cam, tiles in cases:
        gs = gpu_scene(scene)
        comp = oracle.compact(scene) if mode == "roofgs" else None
        flag_sets = [0] if mode == "exact" else [0, binding.RG_FLAG_QUAD_PIXEL]
        for fl in flag_sets:
            img, st = render(gs, cam, mode, flags=fl, stats=True, tile=tile)
            assert st["tiles_x"] == (cam.width + tile[0] - 1) // tile[0]
            assert st["n_entries"] == _keys_equal(gs, scene, cam, om, comp, tile=tile)
            check_view(img, scene, cam, mode, tile=tile, tiles=tiles, comp=comp, max_flagged=0.02,
                       label="%s %s" % (mode, tile))
            # the timed (non-counting) launch gives the same image
            assert np.array_equal(img, render(gs, cam, mode, flags=fl, tile=tile))
        gs.check()


@pytest.mark.parametrize("wh,tile", [((8000, 128), (16, 16)), ((4000, 128), (8, 32))])
def test_tile_rows_wider_than_256_tiles(wh, tile):
    """Wide, flat Gaussians whose tile rows span more than 256 tiles: the front end's count of the
    sort's low tile digit then takes full cycles of 256 besides runs that wrap past digit 255 (500
    tiles per row: rows start at different low digits). Keys, values and ranges bit-exact against
    the oracle (a wrong digit count misplaces entries)."""
    base = small_random_scene(3000, seed=11, spread=1.0)
    wide = single_scene(means=[[0.0, 0.0, 0.0], [0.4, 0.0, 0.5], [-0.3, 0.0, -0.5]],
                        scales=[[1.2, 0.02, 0.02], [2.0, 0.03, 0.02], [0.8, 0.01, 0.05]],
                        quats=[[1.0, 0.0, 0.0, 0.0]] * 3, opac=[0.9, 0.6, 0.95], dc=[[0.8, 0.2, 0.1]] * 3)
    sc = synth.Scene(*(np.concatenate([getattr(base, f), getattr(wide, f)])
                       for f in ("means", "scales", "quats", "opacities", "sh")))
    cam = synth.tiny_camera(*wh)
    gs = gpu_scene(sc)
    comp = oracle.compact(sc)
    _, st = render(gs, cam, "roofgs", stats=True, tile=tile)
    assert st["sort_passes"] == 2  # the front end counts the digits of both passes
    bins = oracle.keys(sc, cam, oracle.ROOFGS, comp=comp, tile=tile)[3]
    assert (bins[-3:, 0] == 1).all() and (bins[-3:, 3] - bins[-3:, 1] + 1 > 256).all()
    assert st["n_entries"] == _keys_equal(gs, sc, cam, oracle.ROOFGS, comp, tile=tile)
    gs.check()


def test_unsupported_tile_shape_is_rejected():
    sc, cams = synth.workload("tiny_256")
    gs = gpu_scene(sc)
    with pytest.raises(binding.RgError) as e:
        gs.render(cams[0], tile=(16, 8))
    assert e.value.status == 8


def test_input_permutation_invariance():
    """Permuting the input Gaussians changes nothing but the index tie-break, in both modes:
    the same sorted keys, the same Gaussians in every run of equal keys (tiles and FP32 or
    quantized depths that tie), and images that differ only where tied Gaussians overlap."""
    sc = synth.clustered_scene(100_000, seed=8)
    cam = synth.orbit_camera(2, 640, 360)
    perm = np.random.default_rng(1).permutation(sc.n)
    ga, gb = gpu_scene(sc), gpu_scene(sc.subset(perm))
    for mode in ("exact", "roofgs"):
        # checked renders: the workspaces grow to the frame's entries
        a, b = render(ga, cam, mode, stats=True)[0], render(gb, cam, mode, stats=True)[0]
        kt = np.uint64 if mode == "exact" else np.uint32
        ka = ga.inspect(binding.RG_INSPECT_KEYS).view(kt)
        kb = gb.inspect(binding.RG_INSPECT_KEYS).view(kt)
        va = ga.inspect(binding.RG_INSPECT_VALUES)
        vb = perm[gb.inspect(binding.RG_INSPECT_VALUES)].astype(np.uint32)  # back to original indices
        assert np.array_equal(ka, kb), mode
        oa, ob = np.lexsort((va, ka)), np.lexsort((vb, kb))
        assert np.array_equal(va[oa], vb[ob]), mode
        # the tie-break can reorder Gaussians only within runs of equal keys: outside the tiles
        # that hold such a run the images are identical
        shift = 32 if mode == "exact" else ga.render(cam, mode=mode, stats=True)[1]["b_d"]
        tied = np.unique((ka[1:][ka[1:] == ka[:-1]].astype(np.uint64) >> np.uint64(shift)).astype(np.int64))
        lay = oracle.layout(cam)
        free = np.ones((cam.height, cam.width), bool)
        for t in tied:
            tx, ty = t % lay["tiles_x"], t // lay["tiles_x"]
            free[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = False
        assert np.array_equal(a[:, free], b[:, free]), (mode, len(tied))
    ga.check()
    gb.check()


@pytest.mark.parametrize("mode", ["exact", "roofgs"])
def test_render_into_pinned_host_memory(mode):
    """out may be pinned host memory that the GPU addresses: the image is written straight
    to the host and equals the device-buffer render."""
    sc, cams = synth.workload("tiny_256")
    gs = gpu_scene(sc)
    dev = gs.render(cams[0], mode=mode)
    host = torch.empty((3, 256, 256), dtype=torch.float32, pin_memory=True)
    gs.render(cams[0], mode=mode, out=host)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)
    gs.check()


# ---------------------------------------------------------------------------
# the row-bucketed front end (default) against the fused front end with the ordered
# allocation (RG_FLAG_ORDERED_FRONT_END): the same entries per tile in the same order
# ---------------------------------------------------------------------------

def _entries(gs):
    return tuple(gs.inspect(w) for w in (binding.RG_INSPECT_KEYS, binding.RG_INSPECT_VALUES,
                                         binding.RG_INSPECT_RANGES))


def _both_front_ends(gs, cam, flags=0, tile=(16, 16)):
    ia, sa = render(gs, cam, "roofgs", flags=flags, stats=True, tile=tile)
    ea = _entries(gs)
    ib, sb = render(gs, cam, "roofgs", flags=flags | binding.RG_FLAG_ORDERED_FRONT_END, stats=True, tile=tile)
    eb = _entries(gs)
    for f in ("n_entries", "n_visible", "n_front", "n_pairs", "n_blends"):
        assert sa[f] == sb[f], (f, sa[f], sb[f])
    for x, y in zip(ea, eb):
        assert np.array_equal(x, y)
    assert np.array_equal(ia, ib)
    return sa, sb


@pytest.mark.parametrize("name", ["tiny_256", "clustered_1080p", "clustered_4k"])
def test_row_buckets_equal_the_ordered_front_end(name):
    """Keys, values and ranges (rebuilt in tile-id order), counters and images (2 and 4 pixels
    per thread) bit-identical between the two front ends; the row-bucketed frame leaves one
    8-bit pass (the tile column) to the sort."""
    sc, cams = synth.workload(name)
    gs = gpu_scene(sc, per_gauss=True)
    cam = cams[0] if name != "clustered_4k" else cams[11]
    for flags in (0, binding.RG_FLAG_QUAD_PIXEL):
        sa, sb = _both_front_ends(gs, cam, flags)
        assert sa["sort_passes"] == 1
        assert sb["sort_passes"] == (sa["b_t"] + 7) // 8
    gs.check()


@pytest.mark.parametrize("wh,hfov,tile", [((4096, 48), 40.0, (16, 16)), ((48, 4096), 0.5, (16, 16)),
                                          ((1000, 700), 60.0, (8, 32)), ((100, 37), 60.0, (16, 16)),
                                          ((1, 1), 60.0, (16, 16))])
def test_row_buckets_extreme_grids_against_the_oracle(wh, hfov, tile):
    """256 tile columns (the key's high byte full), 256 tile rows (the search for the last row's
    end carries into the next column), an 8 x 32 tile grid and ragged images: keys, values and
    ranges bit-exact against the oracle, and equal to the ordered front end's."""
    sc = small_random_scene(4000, seed=5, spread=1.0)
    cam = synth.look_at_camera((0.0, 0.0, -3.0), wh[0], wh[1], hfov, 0.2, 6.0, bg=(0.1, 0.2, 0.3))
    gs = gpu_scene(sc)
    comp = oracle.compact(sc)
    sa, _ = _both_front_ends(gs, cam, tile=tile)
    render(gs, cam, "roofgs", stats=True, tile=tile)
    assert sa["n_entries"] == _keys_equal(gs, sc, cam, oracle.ROOFGS, comp, tile=tile)
    if wh[0] * wh[1] > 1:
        assert sa["n_entries"] > 0
    if wh == (48, 4096):  # entries in the last tile row
        r = gs.inspect(binding.RG_INSPECT_RANGES).reshape(-1, 2)
        assert (r[-3:, 1] > r[-3:, 0]).any()
    gs.check()


def test_row_buckets_capacity_overflow_regrows():
    """A workspace too small for the frame: the row-bucketed front end keeps the entries whose
    slot in its (tile row, depth code, index, tile column) order lies below the capacity, the
    sort covers exactly those (digits recounted from the stored keys), the overflow is
    reported, and the re-rendered frame equals a full one."""
    sc, cams = synth.workload("tiny_256")
    cam = cams[0]
    ref = render(gpu_scene(sc), cam, "roofgs")
    small = gpu_scene(sc)
    small.reserve(1000)
    small.render(cam)
    torch.cuda.synchronize()
    gk = small.inspect(binding.RG_INSPECT_KEYS).view(np.uint32).astype(np.uint64)
    gv = small.inspect(binding.RG_INSPECT_VALUES)
    k, v, _, _ = oracle.keys(sc, cam, oracle.ROOFGS, comp=oracle.compact(sc))
    lay = oracle.layout(cam)
    b_d = np.uint64(lay["b_d"])
    tile = k >> b_d
    tx, ty = tile % np.uint64(lay["tiles_x"]), tile // np.uint64(lay["tiles_x"])
    assert 0 < gk.size < k.size
    kept = np.lexsort((tx, v, k & ((np.uint64(1) << b_d) - np.uint64(1)), ty))[: gk.size]
    expect = kept[np.lexsort((v[kept], k[kept]))]
    assert np.array_equal(gk, k[expect]) and np.array_equal(gv, v[expect])
    with pytest.raises(binding.RgError) as e:
        small.check()
    assert e.value.status == 4
    img, st = render(small, cam, "roofgs", stats=True)
    assert st["regrown"] == 1 and st["capacity"] >= st["n_entries"]
    assert np.array_equal(img, ref)
    small.check()
