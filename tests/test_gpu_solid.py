"""Opaque-triangle render against the oracle's solid render (the sigma -> 0, o = 1
limit of the splat render): winning triangle per pixel exactly and colours within
1e-4 on every pixel outside the FP32 band; a scene over several views and ragged sizes."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth
from gpu_util import UNRESOLVED_CAP

pytestmark = pytest.mark.gpu


def _gpu_solid(scene, cams):
    import torch
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    imgs = new_images(cams)
    ids = [torch.empty((c.H, c.W), dtype=torch.int32, device="cuda") for c in cams]
    ctx.render_solid(st, cams, imgs, ids)
    ctx.check()
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in imgs], [x.cpu().numpy() for x in ids], ctx


@pytest.mark.parametrize("seed,W,H", [(52, 120, 90), (53, 37, 61), (54, 257, 129)])
def test_solid_matches_oracle(seed, W, H):
    scene = synth.random_scene(1500, seed=seed, deg=2, size=(0.05, 0.7), opacity=(0.01, 0.9), sigma=(0.3, 3.0))
    cam = synth.camera_identity(W, H)
    cam.bg = np.array([0.2, 0.1, 0.05], np.float32)
    imgs, ids, _ = _gpu_solid(scene, [cam])
    ref = O.render_solid(scene, cam)
    ok = ref["flags"] == 0
    print(f"[flagged] solid {W}x{H}: {int((~ok).sum())} of {ok.size} pixels")
    assert (~ok).sum() <= UNRESOLVED_CAP * ok.size
    np.testing.assert_array_equal(ids[0][ok], ref["id"][ok])
    np.testing.assert_allclose(imgs[0][:, ok], ref["image"][:, ok], atol=1e-4)


def test_solid_multiview_and_no_backward():
    from paper_2505_19175_gb300.native import TriError
    scene = synth.random_scene(900, seed=55, deg=1, size=(0.05, 0.6))
    cams = [synth.camera_identity(96, 72), synth.camera_look_at((0.3, -0.1, -0.4), (0, 0, 3.5), 64, 80)]
    imgs, ids, ctx = _gpu_solid(scene, cams)
    for v, cam in enumerate(cams):
        ref = O.render_solid(scene, cam)
        ok = ref["flags"] == 0
        print(f"[flagged] solid view {v}: {int((~ok).sum())} of {ok.size} pixels")
        assert (~ok).sum() <= UNRESOLVED_CAP * ok.size
        np.testing.assert_array_equal(ids[v][ok], ref["id"][ok])
        np.testing.assert_allclose(imgs[v][:, ok], ref["image"][:, ok], atol=1e-4)
    import torch
    with pytest.raises(TriError):
        ctx.render_bwd([torch.zeros((3, c.H, c.W), device="cuda") for c in cams])
