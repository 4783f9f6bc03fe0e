"""The allocation-free forward render agrees with the regular entry points.

Callers that cannot allocate device memory (a plugin inside an application that owns
the device allocator, a loop that reserved all memory up front) render through
tri_render_fwd_noalloc, whose workspace is a fixed array inside the library. This test
calls it through the C ABI twice in a row, on two different scenes and image sizes (the
second smaller, so stale contents of the shared array would show), and compares each
result with tri_preprocess + tri_bin_sort + tri_render_fwd within the image tolerance
of the other tests. It runs last so that a failure here never hides another test."""
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


def _render_noalloc(scene, cam):
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
    assert int(status.item()) == 0
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
