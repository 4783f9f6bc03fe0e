"""The forward fused with the L1 loss (tri_render_fwd_l1) against the forward followed
by the separate loss kernel on the views' images as one array: images and gradients
bit for bit, the loss up to summation order; inside a captured step; and refused with
the per-pixel sort."""
import numpy as np
import pytest

from paper_2505_19175_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(seed=95):
    from paper_2505_19175_gb300.renderer import Context, SceneTensors
    scene = synth.random_scene(900, seed=seed, deg=2, size=(0.05, 0.6))
    cams = [synth.camera_identity(96, 72), synth.camera_look_at((0.3, -0.1, -0.4), (0, 0, 3.5), 61, 45)]
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    ctx.preprocess(st, cams)
    ctx.bin_sort(sync=True)
    return ctx, st, cams


def test_fused_l1_matches_the_separate_loss():
    import torch
    from paper_2505_19175_gb300.renderer import new_images, loss_l1
    ctx, st, cams = _setup()
    tg = [torch.as_tensor(synth.target_image(c.H, c.W, seed=7 + k)).cuda() for k, c in enumerate(cams)]
    ref = new_images(cams)
    ctx.render_fwd(ref)
    loss_ref, g_ref = loss_l1(torch.cat([x.reshape(-1) for x in ref]), torch.cat([x.reshape(-1) for x in tg]))
    imgs = new_images(cams)
    grads = [torch.empty_like(x) for x in imgs]
    loss = torch.empty((), device="cuda")
    ctx.render_fwd_l1(imgs, tg, grads, loss)
    ctx.check()
    torch.cuda.synchronize()
    for a, b in zip(imgs, ref):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    torch.testing.assert_close(torch.cat([x.reshape(-1) for x in grads]), g_ref, rtol=0, atol=0)
    assert abs(float(loss) - float(loss_ref)) <= 1e-5 * float(loss_ref)
    # some pixels carry each sign
    g = torch.cat([x.reshape(-1) for x in grads])
    assert (g > 0).any() and (g < 0).any()


def test_fused_l1_in_a_captured_step():
    import torch
    from paper_2505_19175_gb300.renderer import new_images
    ctx, st, cams = _setup(96)
    ctx.reserve(int(ctx.bin_sort(sync=True) * 1.5) + 1024)
    tg = [torch.as_tensor(synth.target_image(c.H, c.W, seed=11 + k)).cuda() for k, c in enumerate(cams)]
    imgs = new_images(cams)
    grads = [torch.empty_like(x) for x in imgs]
    loss = torch.empty((), device="cuda")
    dv, dsh = torch.empty_like(st.verts), torch.empty_like(st.sh)
    do, ds = torch.empty_like(st.opacity), torch.empty_like(st.sigma)

    def step():
        ctx.preprocess(st, cams)
        ctx.bin_sort(sync=False)
        ctx.render_fwd_l1(imgs, tg, grads, loss)
        ctx.render_bwd(grads)
        ctx.preprocess_bwd(dv, dsh, do, ds)

    step()
    torch.cuda.synchronize()
    want = [x.clone() for x in (*grads, loss, dv, do)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        got = (*grads, loss, dv, do)
        for x, y in zip(got[:2], want[:2]):
            torch.testing.assert_close(x, y, rtol=0, atol=0)
        torch.testing.assert_close(got[2], want[2], rtol=1e-5, atol=0)
        for x, y in zip(got[3:], want[3:]):
            torch.testing.assert_close(x, y, rtol=1e-5, atol=1e-6 * float(y.abs().max()))


def test_fused_l1_needs_the_tile_sort():
    import torch
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.native import TriError
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    scene = synth.random_scene(200, seed=97, deg=0)
    cam = synth.camera_identity(48, 32)
    ctx = Context()
    ctx.set_sort(N.SORT_PIXEL)
    ctx.preprocess(SceneTensors.from_numpy(scene), [cam])
    ctx.bin_sort(sync=True)
    imgs = new_images([cam])
    with pytest.raises(TriError):
        ctx.render_fwd_l1(imgs, [torch.zeros_like(imgs[0])], [torch.empty_like(imgs[0])])
