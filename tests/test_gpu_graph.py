"""A fwd+bwd step captured as a CUDA graph replays to the eager step's results."""
import numpy as np
import pytest

from paper_2505_19175_gb300 import synth

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_step():
    import torch
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images, loss_l1
    scene = synth.random_scene(3000, seed=41, deg=3, size=(0.05, 0.5))
    cam = synth.camera_identity(300, 200)
    st = SceneTensors.from_numpy(scene)
    tgt = torch.as_tensor(synth.target_image(cam.H, cam.W, seed=3)).cuda()
    ctx = Context()
    ctx.preprocess(st, [cam])
    n = ctx.bin_sort(sync=True)
    ctx.reserve(int(n * 1.5) + 64)
    img = new_images([cam])
    outs = [torch.empty_like(x) for x in (st.verts, st.sh, st.opacity, st.sigma)]

    def step():
        ctx.preprocess(st, [cam])
        ctx.bin_sort(sync=False)
        ctx.render_fwd(img)
        _, g = loss_l1(img[0], tgt)
        ctx.render_bwd([g])
        ctx.preprocess_bwd(*outs)

    step()
    torch.cuda.synchronize()
    eager_img = img[0].clone()
    eager = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    img[0].zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    ctx.check()
    assert torch.equal(img[0], eager_img)
    for a, b in zip(outs, eager):
        # atomics make the gradient sums order-dependent at the rounding level
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()))
