"""Pruning statistics of the forward render (Sec. 3.3 "Pruning") against the oracle:
per (view, triangle) composited-pixel counts exactly and the largest blending weight
T o within FP32 rounding, for every triangle none of whose pixels is in the FP32 band."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_stats(scene, cams):
    import torch
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    ctx.preprocess(st, cams)
    ctx.bin_sort(sync=True)
    imgs = new_images(cams)
    n = scene.n * len(cams)
    mw = torch.full((n,), -1.0, device="cuda")
    npx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ctx.render_fwd(imgs, stats=(mw, npx))
    ctx.check()
    torch.cuda.synchronize()
    return mw.cpu().numpy().reshape(len(cams), -1), npx.cpu().numpy().reshape(len(cams), -1), imgs


@pytest.mark.parametrize("seed", [31, 32])
def test_stats_match_oracle(seed):
    scene = synth.random_scene(1200, seed=seed, deg=2, size=(0.05, 0.7), opacity=(0.05, 0.95))
    cams = [synth.camera_identity(120, 90), synth.camera_look_at((0.4, -0.2, -0.3), (0, 0, 3.5), 96, 80)]
    mw, npx, _ = _gpu_stats(scene, cams)
    for v, cam in enumerate(cams):
        ref = O.render_stats(scene, cam)
        ok = ref["amb"] == 0
        # a triangle in a pixel with a decision in the FP32 band may gain or lose that pixel
        n_flag = int(((O.render(scene, cam, flags=True)["flags"] & np.uint8(0xFF ^ O.AMB_GRAD)) != 0).sum())
        print(f"[flagged] stats view {v}: {int((~ok).sum())} of {ok.size} triangles in {n_flag} flagged pixels")
        assert ok.mean() >= 0.99
        np.testing.assert_array_equal(npx[v][ok], ref["n_pix"][ok])
        np.testing.assert_allclose(mw[v][ok], ref["max_weight"][ok], rtol=2e-5, atol=1e-6)
        assert np.all(np.abs(npx[v][~ok].astype(np.int64) - ref["n_pix"][~ok]) <= n_flag)
        # every triangle, flagged or not, has consistent outputs
        assert np.all((npx[v] > 0) == (mw[v] > 0))


def test_stats_leave_the_image_unchanged_and_drive_pruning():
    import torch
    from paper_2505_19175_gb300 import prune
    from gpu_util import gpu_forward
    scene = synth.random_scene(800, seed=33, deg=1, size=(0.05, 0.6))
    cams = [synth.camera_identity(100, 80), synth.camera_identity(64, 80, cx=50.0, cy=40.0, fx=93.75)]
    mw, npx, imgs = _gpu_stats(scene, cams)
    plain, _, _, _, _ = gpu_forward(scene, cams)
    for v in range(len(cams)):
        np.testing.assert_array_equal(imgs[v].cpu().numpy(), plain[v].astype(np.float32))
    refs = [O.render_stats(scene, c) for c in cams]
    amb = np.any([r["amb"] != 0 for r in refs], axis=0)
    ref_keep = O.prune_keep(np.stack([r["max_weight"] for r in refs]), np.stack([r["n_pix"] for r in refs]), 0.05)
    ps = prune.PruneStats(scene.n, device="cuda")
    ps.update(torch.as_tensor(mw).cuda(), torch.as_tensor(npx).cuda())
    keep = ps.keep(0.05).cpu().numpy()
    np.testing.assert_array_equal(keep[~amb], ref_keep[~amb])
    assert 0 < keep.sum() < scene.n


def test_pruning_rule_on_the_device_folds_batches_of_views():
    """tri_prune_fold over batches of 3, 1 and 3 views, then tri_prune_mask, decides as
    the oracle's rule over all seven views at once (weights compared in FP32 on both
    sides: the statistics are FP32)."""
    import torch
    from paper_2505_19175_gb300 import prune
    rng = np.random.default_rng(8)
    V, n = 7, 5000
    mw = (rng.uniform(0, 1, (V, n)) * (rng.uniform(size=(V, n)) < 0.6)).astype(np.float32)
    npix = rng.integers(0, 4, (V, n)).astype(np.int32)
    want = O.prune_keep(mw, npix, tau_prune=np.float32(0.5), min_views=3)
    ps = prune.PruneStats(n, device="cuda")
    for a, b in ((0, 3), (3, 4), (4, 7)):
        ps.update(torch.as_tensor(mw[a:b]).cuda().reshape(-1), torch.as_tensor(npix[a:b]).cuda().reshape(-1))
    np.testing.assert_array_equal(ps.keep(0.5, min_views=3).cpu().numpy(), want)
    np.testing.assert_array_equal(ps.max_weight.cpu().numpy(), mw.max(0))
    np.testing.assert_array_equal(ps.views.cpu().numpy(), (npix >= 2).sum(0))
    whole = prune.keep_mask(torch.as_tensor(mw).cuda(), torch.as_tensor(npix).cuda(), 0.5, 3)
    np.testing.assert_array_equal(whole.cpu().numpy(), want)
    assert 0 < want.sum() < n
    ps.reset()
    assert not ps.keep(0.0, min_views=1).any()
    # ragged: one triangle, no views
    one = prune.PruneStats(1, device="cuda")
    one.update(torch.zeros(0, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert not one.keep(0.0, min_views=1).any()
