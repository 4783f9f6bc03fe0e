"""Failure handling without faulting the GPU: host-side injection (TRI_FAULT) of a
failed device allocation and of slow requests. Calls return clean error codes, the
context keeps working, and the server keeps serving."""
import numpy as np
import pytest

from paper_2505_19175_gb300 import synth

pytestmark = pytest.mark.gpu


def _scene_cam():
    return synth.random_scene(300, seed=81, deg=1), synth.camera_identity(64, 48)


def _render(ctx, st, cam):
    import torch
    from paper_2505_19175_gb300.renderer import new_images
    ctx.preprocess(st, [cam])
    ctx.bin_sort(sync=True)
    img = new_images([cam])
    ctx.render_fwd(img)
    ctx.check()
    torch.cuda.synchronize()
    return img[0].cpu().numpy()


def test_failed_allocation_is_reported_and_the_context_recovers(monkeypatch):
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import Context, SceneTensors
    scene, cam = _scene_cam()
    st = SceneTensors.from_numpy(scene)
    monkeypatch.setenv("TRI_FAULT", "alloc:3")
    ctx = Context()
    monkeypatch.delenv("TRI_FAULT")
    with pytest.raises(N.TriError) as e:
        _render(ctx, st, cam)
    assert e.value.status == N.TRI_ERR_OOM
    # the next calls allocate normally and give the same image as a fresh context
    np.testing.assert_array_equal(_render(ctx, st, cam), _render(Context(), st, cam))


def test_server_keeps_serving_after_a_failed_allocation(monkeypatch):
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.serve import Server
    scene, cam = _scene_cam()
    monkeypatch.setenv("TRI_FAULT", "alloc:2")
    srv = Server(max_batch=1, slots=1)
    monkeypatch.delenv("TRI_FAULT")
    sid = srv.add_scene(scene)
    codes = []
    for _ in range(3):
        t, _ = srv.submit(sid, cam)
        codes.append(srv.wait(t))
    assert codes[0] == N.TRI_ERR_OOM and codes[1:] == [0, 0]
    st = srv.stats()
    assert st["completed"] == 2 and st["rejected"] == 1
    srv.close()


def test_slow_requests_time_out_and_the_server_recovers(monkeypatch):
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.serve import Server
    scene, cam = _scene_cam()
    monkeypatch.setenv("TRI_FAULT", "slow:40")
    srv = Server(max_batch=1, slots=1, timeout_ms=10)
    monkeypatch.delenv("TRI_FAULT")
    sid = srv.add_scene(scene)
    tickets = [srv.submit(sid, cam)[0] for _ in range(8)]
    codes = [srv.wait(t) for t in tickets]
    assert codes[0] == 0 and N.TRI_ERR_TIMEOUT in codes and set(codes) <= {0, N.TRI_ERR_TIMEOUT}
    t, _ = srv.submit(sid, cam)          # alone in the queue: within its deadline again
    assert srv.wait(t) == 0
    srv.close()


def test_bounded_device_wait_gives_up_and_the_context_recovers():
    """A scan CTA whose predecessor's look-back word nothing sets: its wait gives up
    after the (shortened) limit, the kernel finishes, tri_ctx_check reports
    TRI_ERR_TIMEOUT, and the next normal call on the same context renders the image the
    oracle computes."""
    import time
    import torch
    import oracle as O
    from gpu_util import check_image
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    scene = synth.random_scene(2000, seed=82, deg=1, size=(0.05, 0.4))
    cam = synth.camera_identity(640, 480, fx=600.0)     # 1,200 tiles: two scan CTAs
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    img = new_images([cam])
    ctx.preprocess(st, [cam])
    ctx.debug_withhold_scan(cta=0, wait_ns=2_000_000)   # CTA 1 waits on a word nothing sets
    t0 = time.perf_counter()
    ctx.bin_sort(sync=False)
    ctx.render_fwd(img)
    with pytest.raises(N.TriError) as e:
        ctx.check()
    waited = time.perf_counter() - t0
    assert e.value.status == N.TRI_ERR_TIMEOUT
    assert waited < 0.5                                  # the 2 ms limit, not the 1 s default
    # the same context, a normal run
    T = [torch.empty((cam.H, cam.W), device="cuda")]
    ctx.preprocess(st, [cam])
    ctx.bin_sort(sync=True)
    ctx.render_fwd(img, T)
    ctx.check()
    torch.cuda.synchronize()
    ref = O.render(scene, cam, flags=True)
    check_image(img[0].cpu().numpy().astype(np.float64), T[0].cpu().numpy().astype(np.float64), ref,
                label="after a wait gave up")
