"""Scene checkpoints round-trip exactly (host side, no GPU)."""
import numpy as np
import pytest

from paper_2505_19175_gb300 import scene_io, synth


def test_round_trip(tmp_path):
    s = synth.random_scene(123, seed=3, deg=3)
    p = str(tmp_path / "scene.npz")
    scene_io.save(p, s)
    t = scene_io.load(p)
    for k in ("verts", "sh", "opacity", "sigma"):
        np.testing.assert_array_equal(getattr(t, k), getattr(s, k).astype(np.float32))
    assert t.sh_degree == 3 and t.n == 123
    assert t.verts.size + t.sh.size + t.opacity.size + t.sigma.size == 59 * 123


def test_inconsistent_file_is_rejected(tmp_path):
    p = str(tmp_path / "bad.npz")
    np.savez(p, verts=np.zeros((4, 3, 3), np.float32), sh=np.zeros((4, 1, 3), np.float32),
             opacity=np.zeros(3, np.float32), sigma=np.zeros(4, np.float32), sh_degree=np.int32(0))
    with pytest.raises(ValueError):
        scene_io.load(p)
