"""Seeded synthetic inputs: generator definition and determinism."""
import os

import numpy as np

from paper_2103_10765_gb300 import synth
from conftest import GOLDEN


def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        vals = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#") and not ln.startswith("seed")]
    want = [int(v, 16) for v in vals]
    assert synth.splitmix64_scalar(0, 3) == want
    assert [int(v) for v in synth.splitmix64(0, 3)] == want


def test_vectorised_matches_scalar_with_offset():
    s = synth.splitmix64_scalar(987654321, 50)
    v = synth.splitmix64(987654321, 20, start=30)
    assert [int(x) for x in v] == s[30:]


def test_uniform_range_and_normal_moments():
    u = synth.uniforms(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    n = synth.normals(8, 200001)
    assert n.shape == (200001,)
    assert abs(n.mean()) < 0.01 and abs(n.std() - 1.0) < 0.01


def test_scene_deterministic_and_clamped():
    a = synth.clean_scene(96, 80, 2)
    b = synth.clean_scene(96, 80, 2)
    c = synth.clean_scene(96, 80, 3)
    assert a.dtype == np.float32 and a.shape == (96, 80)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0


def test_noise_level():
    clean, noisy = synth.make_pair(256, 256, 25 / 255, 1)
    d = noisy.astype(np.float64) - clean
    assert abs(d.std() - 25 / 255) < 0.003
    assert noisy.dtype == np.float32


def test_empty():
    assert synth.clean_scene(0, 5, 1).shape == (0, 5)
