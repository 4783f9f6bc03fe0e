"""The allocation-free forward render agrees with the regular entry points.

Callers that cannot allocate device memory (a plugin inside an application that owns
the device allocator, a loop that reserved all memory up front) render through
tri_render_fwd_noalloc, whose workspace is a fixed array inside the library. This test
calls it through the C ABI twice in a row, on two different scenes and image sizes (the
second smaller, so stale contents of the shared array would show), and compares each
result with tri_preprocess + tri_bin_sort + tri_render_fwd within the image tolerance
of the other tests; and the paths where leftovers of an earlier call could show: an
empty scene, a larger image after a smaller one, and a pair list beyond the array's
limit. It runs last so that a failure here never hides another test."""
import ctypes as C

import numpy as np
import pytest

from paper_2505_19175_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _noalloc_fn():
    from paper_2505_19175_gb300 import native as N
    f = N.lib().tri_render_fwd_noalloc
    f.argtypes = [C.POINTER(N.tri_scene), C.POINTER(N.tri_camera), C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def _render_noalloc(scene, cam, want_status=0):
    import torch
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import SceneTensors
    st = SceneTensors.from_numpy(scene)
    img = torch.full((3, cam.H, cam.W), float("nan"), device="cuda")
    T = torch.empty((cam.H, cam.W), device="cuda")
    nc = torch.empty((cam.H, cam.W), device="cuda", dtype=torch.int32)
    status = torch.full((1,), -1, device="cuda", dtype=torch.int32)
    abi_scene = st.as_abi()
    abi_cam = N.make_camera(cam)
    rc = _noalloc_fn()(C.byref(abi_scene), C.byref(abi_cam), img.data_ptr(), T.data_ptr(), nc.data_ptr(),
                       status.data_ptr(), int(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    assert int(status.item()) == want_status
    return img.cpu().numpy(), T.cpu().numpy(), nc.cpu().numpy()


def test_noalloc_matches_regular_path_on_two_calls():
    from gpu_util import gpu_forward
    cases = [(synth.random_scene(4000, seed=51, deg=3, size=(0.05, 0.6), sigma=(0.3, 3.0)),
              synth.camera_look_at((0.2, -0.1, -0.4), (0.0, 0.0, 3.5), 320, 240)),
             (synth.random_scene(1500, seed=52, deg=1, size=(0.05, 0.5)), synth.camera_identity(200, 150))]
    for scene, cam in cases:
        img, T, nc = _render_noalloc(scene, cam)
        ref_img, ref_T, ref_nc, _, _ = gpu_forward(scene, [cam])
        assert np.isfinite(img).all()
        np.testing.assert_allclose(img, ref_img[0], rtol=0, atol=TOL)
        np.testing.assert_allclose(T, ref_T[0], rtol=0, atol=TOL)
        np.testing.assert_array_equal(nc, ref_nc[0])


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2505_19175_gb300 import native as N
    scene = synth.random_scene(8, seed=53, deg=0)
    big = synth.camera_identity(4096, 4096)   # above the pixel limit
    import torch
    from paper_2505_19175_gb300.renderer import SceneTensors
    st = SceneTensors.from_numpy(scene)
    img = torch.empty(1, device="cuda")
    rc = _noalloc_fn()(C.byref(st.as_abi()), C.byref(N.make_camera(big)), img.data_ptr(), None, None, None,
                       int(torch.cuda.current_stream().cuda_stream))
    assert rc == N.TRI_ERR_CAPACITY


def test_noalloc_empty_scene_larger_image_and_pair_overflow():
    from gpu_util import gpu_forward
    # a scene first, so that the array holds ranges, records and pairs
    scene = synth.random_scene(3000, seed=54, deg=2, size=(0.05, 0.5))
    small = synth.camera_identity(160, 120)
    _render_noalloc(scene, small)
    # no triangles: the background everywhere, T = 1, no fragments
    cam = synth.camera_identity(300, 200)
    cam.bg = np.array([0.1, 0.2, 0.3], np.float32)
    img, T, nc = _render_noalloc(synth.random_scene(0, seed=0, deg=0), cam)
    np.testing.assert_array_equal(img, np.broadcast_to(cam.bg[:, None, None], img.shape))
    assert np.all(T == 1.0) and np.all(nc == 0)
    # a larger image (more tiles) after the smaller ones
    big = synth.camera_identity(1024, 768, fx=640.0)
    img, T, nc = _render_noalloc(scene, big)
    ref_img, ref_T, ref_nc, _, _ = gpu_forward(scene, [big])
    np.testing.assert_allclose(img, ref_img[0], rtol=0, atol=TOL)
    np.testing.assert_allclose(T, ref_T[0], rtol=0, atol=TOL)
    np.testing.assert_array_equal(nc, ref_nc[0])
    # large triangles over a 2048 x 1088 image: more pairs than the array holds; the
    # overflow is reported (status bit 2), the image stays finite
    huge = synth.random_scene(5000, seed=55, deg=0, size=(0.4, 0.9))    # ~2.4M pairs
    full = synth.camera_identity(2048, 1088, fx=1920.0)
    img, T, nc = _render_noalloc(huge, full, want_status=4)
    assert np.isfinite(img).all() and np.isfinite(T).all()
    # and the next call within the limits is clean again
    img, T, nc = _render_noalloc(scene, small)
    ref_img, _, _, _, _ = gpu_forward(scene, [small])
    np.testing.assert_allclose(img, ref_img[0], rtol=0, atol=TOL)
