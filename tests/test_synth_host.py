"""Seeded input generators (host only): determinism and the pruning stand-in."""
from __future__ import annotations

import numpy as np

from paper_2608_15785_gb300 import synth


def test_generators_are_seeded():
    a, b = synth.clustered_scene(5000, 3), synth.clustered_scene(5000, 3)
    for f in ("means", "scales", "quats", "opacities", "sh"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.means, synth.clustered_scene(5000, 4).means)


def test_prune_by_footprint_keeps_the_largest_scores_in_order():
    sc = synth.clustered_scene(20_000, 1)
    pr = synth.prune_by_footprint(sc, 0.1)
    assert pr.n == 2000
    s = np.sort(sc.scales, axis=1)
    score = sc.opacities * s[:, 2] * s[:, 1]
    # the kept Gaussians are exactly the 2000 best scores, in their original order
    kept = np.flatnonzero(np.isin(sc.means.view([("", sc.means.dtype)] * 3).ravel(),
                                  pr.means.view([("", pr.means.dtype)] * 3).ravel()))
    assert kept.size == 2000
    assert np.array_equal(sc.means[kept], pr.means)
    dropped = np.setdiff1d(np.arange(sc.n), kept)
    assert score[kept].min() >= score[dropped].max()
