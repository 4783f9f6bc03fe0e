"""Serving: continuous batching of mixed-resolution requests returns, for each request,
the same image as rendering it alone; admission by memory, deadlines and a pair-list
overflow give clean statuses and the server keeps serving."""
import numpy as np
import pytest

from paper_2505_19175_gb300 import synth

pytestmark = pytest.mark.gpu


def _scene(n=20000, seed=61):
    return synth.scene_shells(n, seed=seed, n_shell=6, r_lo=1.0, r_hi=3.0)


def _alone(scene, cam):
    from gpu_util import gpu_forward
    imgs, _, _, _, _ = gpu_forward(scene, [cam])
    return imgs[0]


def test_each_request_is_the_same_alone_and_in_the_mix():
    from paper_2505_19175_gb300.serve import Server
    scene = _scene()
    reqs = synth.serve_requests(24, seed=62)
    cams = [c for _, _, c in reqs]
    # scale resolutions down so the test stays small
    small = []
    for c in cams:
        W, H = c.W // 4, c.H // 4
        small.append(synth.camera_look_at(c.position(), (0, 0, 0), W, H))
    srv = Server(max_batch=8, slots=3, max_width=1920, max_height=1080, use_graphs=True)
    sid = srv.add_scene(scene)
    tickets = [srv.submit(sid, c) for c in small]
    for t, _ in tickets:
        assert srv.wait(t, 60000) == 0
    # a second pass over the same cameras replays captured graphs
    tickets2 = [srv.submit(sid, c) for c in small]
    for t, _ in tickets2:
        assert srv.wait(t, 60000) == 0
    st = srv.stats()
    assert st["completed"] == 48 and st["mean_batch"] > 1.0
    for (t, out), (t2, out2), c in zip(tickets, tickets2, small):
        ref = _alone(scene, c)
        np.testing.assert_array_equal(out.cpu().numpy(), ref.astype(np.float32))
        np.testing.assert_array_equal(out2.cpu().numpy(), ref.astype(np.float32))
    srv.close()


def test_multiple_scenes_and_removal():
    from paper_2505_19175_gb300.serve import Server
    a, b = _scene(8000, 63), _scene(12000, 64)
    cam = synth.camera_look_at((0.0, -0.5, -4.0), (0, 0, 0), 96, 64)
    srv = Server(max_batch=4, slots=2)
    ia, ib = srv.add_scene(a), srv.add_scene(b)
    ta = [srv.submit(ia, cam) for _ in range(3)]
    tb = [srv.submit(ib, cam) for _ in range(3)]
    for t, _ in ta + tb:
        assert srv.wait(t) == 0
    ra, rb = _alone(a, cam).astype(np.float32), _alone(b, cam).astype(np.float32)
    for _, o in ta:
        np.testing.assert_array_equal(o.cpu().numpy(), ra)
    for _, o in tb:
        np.testing.assert_array_equal(o.cpu().numpy(), rb)
    srv.remove_scene(ia)
    from paper_2505_19175_gb300.native import TriError
    with pytest.raises(TriError):
        srv.submit(ia, cam)
    t, o = srv.submit(ib, cam)
    assert srv.wait(t) == 0
    srv.close()


def _workspace(scene, cam):
    import ctypes as C
    from paper_2505_19175_gb300 import native as N
    sc = N.tri_scene()
    sc.verts = sc.sh = sc.opacity = sc.sigma = 16
    sc.n, sc.sh_degree = scene.n, scene.sh_degree
    b = C.c_size_t()
    N.check(N.lib().tri_workspace_query(C.byref(sc), N.camera_array([cam]), 1, 0, C.byref(b)))
    return int(b.value)


def test_admission_by_memory_budget():
    from paper_2505_19175_gb300.native import TriError
    from paper_2505_19175_gb300.serve import Server
    scene = _scene(20000, 65)
    srv = Server(mem_budget_bytes=2 << 20, max_batch=2, slots=1)   # 2 MB: the scene (4.7 MB) cannot fit
    with pytest.raises(TriError):
        srv.add_scene(scene)
    srv.close()
    big = synth.camera_look_at((0.0, 0.0, -4.0), (0, 0, 0), 1920, 1080)
    small = synth.camera_look_at((0.0, 0.0, -4.0), (0, 0, 0), 64, 48)
    need_big, need_small = _workspace(scene, big), _workspace(scene, small)
    assert need_big > need_small
    nsh = scene.n * scene.sh.shape[1] * 12
    scene_bytes = 256 * (((scene.n * 36 + 255) // 256) + ((nsh + 255) // 256) + 2 * ((scene.n * 4 + 255) // 256))
    srv = Server(mem_budget_bytes=scene_bytes + (need_big + need_small) // 2, max_batch=2, slots=1)
    sid = srv.add_scene(scene)
    t, _ = srv.submit(sid, big)       # its workspace does not fit next to the scene
    assert srv.wait(t) == 4           # TRI_ERR_CAPACITY
    t, _ = srv.submit(sid, small)     # the server keeps serving
    assert srv.wait(t) == 0
    st = srv.stats()
    assert st["rejected"] >= 1 and st["completed"] >= 1
    srv.close()


def test_deadline_and_resolution_limit():
    from paper_2505_19175_gb300.native import TriError
    from paper_2505_19175_gb300.serve import Server
    scene = _scene(20000, 66)
    srv = Server(max_batch=1, slots=1, timeout_ms=1, max_width=640, max_height=480)
    sid = srv.add_scene(scene)
    with pytest.raises(TriError):
        srv.submit(sid, synth.camera_look_at((0, 0, -4.0), (0, 0, 0), 1280, 720))
    cam = synth.camera_look_at((0.0, 0.0, -4.0), (0, 0, 0), 640, 480)
    tickets = [srv.submit(sid, cam) for _ in range(64)]
    codes = [srv.wait(t) for t, _ in tickets]
    st = srv.stats()
    assert st["timed_out"] >= 1 and st["timed_out"] + st["completed"] == 64
    assert set(codes) <= {0, 5}
    srv.close()


def test_pair_overflow_reruns_the_batch():
    """Large triangles give more (tile, item) pairs than the default list holds; the
    server detects the overflow at completion, grows the list and re-runs the batch."""
    from paper_2505_19175_gb300.serve import Server
    rng = np.random.default_rng(67)
    n = 300
    c = np.stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), rng.uniform(3.0, 4.0, n)], 1)
    v = c[:, None, :] + 2.5 * rng.standard_normal((n, 3, 3)) * np.array([1.0, 1.0, 0.05])
    scene = synth.Scene(v.astype(np.float32), (0.2 * rng.standard_normal((n, 1, 3))).astype(np.float32),
                        rng.uniform(0.05, 0.3, n).astype(np.float32), rng.uniform(0.3, 1.0, n).astype(np.float32), 0)
    cam = synth.camera_identity(1920, 1080)
    srv = Server(max_batch=2, slots=1)
    sid = srv.add_scene(scene)
    t, out = srv.submit(sid, cam)
    assert srv.wait(t) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), _alone(scene, cam).astype(np.float32))
    srv.close()


def test_graph_policy_counters():
    """graph_after=2: a composition runs eagerly twice, is captured on its second run
    and replayed from then on; every run gives the same image."""
    from paper_2505_19175_gb300.serve import Server
    scene = _scene(10000, 68)
    cam = synth.camera_look_at((0.0, -0.5, -4.0), (0, 0, 0), 160, 96)
    srv = Server(max_batch=1, slots=1, graph_after=2)
    sid = srv.add_scene(scene)
    outs = []
    for _ in range(4):
        t, o = srv.submit(sid, cam)
        assert srv.wait(t) == 0
        outs.append(o.cpu().numpy())
    st = srv.stats()
    assert st["eager_batches"] == 2 and st["graph_captures"] == 1 and st["graph_replays"] == 2
    assert st["queue_p99_ms"] >= 0.0
    ref = _alone(scene, cam).astype(np.float32)
    for o in outs:
        np.testing.assert_array_equal(o, ref)
    srv.close()
