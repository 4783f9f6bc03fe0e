"""ctypes wrapper of the FP64 C oracle (``trisplat_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's
CPU-baseline leg, never by the product. It shares no code with the CUDA path; the two
meet only in the seeded input generators.

Scenes and cameras are read by key or attribute: a scene has ``verts`` [N,3,3],
``sh`` [N,(d+1)^2,3], ``opacity`` [N], ``sigma`` [N] (any float type; computed in
FP64) and ``sh_degree``; a
camera has ``R`` (3x3, world->camera, OpenCV axes), ``t`` (3), ``fx, fy, cx, cy``,
``W, H`` and ``bg`` (3).

The constants are the readings of the paper's unstated values (Sec. 3.1 defers the
compositing rule to prior splatting work; Supp. "Tile assignment" leaves the cutoff
unset): alpha clamp 0.99, skip below 1/255, stop before transmittance drops below
1e-4, near plane 0.2, degenerate inradius 1e-4 px, 16x16 tiles, and a rectangle pad of
2^-9 px that absorbs FP32 rounding of the tight rectangle. ``EXACT_CONSTS`` switches
the three compositing thresholds off for property and finite-difference tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trisplat_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

DEFAULT_CONSTS = dict(alpha_max=0.99, alpha_min=1.0 / 255.0, t_eps=1e-4, z_near=0.2,
                      r_min=1e-4, tile=16, rect_pad=2.0 ** -9, window=0, sort=0)
WINDOW_POWER, WINDOW_SIGMOID = 0, 1       # Eq. indicator1 (the paper's), Eq. indicator2
# compositing order: per tile by centroid depth (the paper's), or per pixel by the depth
# of the triangle's plane along the pixel's ray (the per-pixel sort of its future work)
SORT_TILE, SORT_PIXEL = 0, 1
EXACT_CONSTS = dict(DEFAULT_CONSTS, alpha_max=1.0, alpha_min=0.0, t_eps=0.0)

AMB_SKIP, AMB_STOP, AMB_ORDER, AMB_SENS, AMB_CULL, AMB_UNRES, AMB_GRAD = 1, 2, 4, 8, 16, 32, 64
AMB_DECISION = AMB_SKIP | AMB_STOP | AMB_ORDER | AMB_CULL
# one listed outcome of a pixel with a decision in the FP32 band (the C record)
ALT_DTYPE = np.dtype([("pix", "<i4"), ("n_kept", "<i4"), ("image", "<f8", (3,)), ("T", "<f8")])

_lock = threading.Lock()
_lib = None


_CHECK_SRC = os.path.join(_HERE, "sanitize_check.c")
_CHECK_EXE = os.path.join(_BUILD, "sanitize_check")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FMA contraction), and the C
    driver of its sanitizer test (built here without the sanitizers, which the test
    adds when it runs it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_CHECK_SRC))
    if force or not os.path.exists(_CHECK_EXE) or os.path.getmtime(_CHECK_EXE) < newest:
        tmp = _CHECK_EXE + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-o", tmp, _CHECK_SRC, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _CHECK_EXE)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_render.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, ctypes.c_int,
                                       P, P, P, P, P, P]
            lib.orc_render_alts.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, ctypes.c_int,
                                            P, P, P, P, P, P, P, ctypes.c_size_t, P]
            lib.orc_render_grad.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P,
                                            P, P, P, P, P, P, P]
            lib.orc_render_solid.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P, P, P, P]
            lib.orc_render_stats.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P, P, P]
            lib.orc_tri_info.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P, P]
            lib.orc_tri2d.argtypes = [P, P]
            lib.orc_window.argtypes = [P, ctypes.c_double, ctypes.c_int, P, P, P]
            lib.orc_window_sigmoid.argtypes = [P, ctypes.c_double, ctypes.c_int, P, P, P]
            lib.orc_sh_eval.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _get(obj, name):
    return obj[name] if isinstance(obj, dict) else getattr(obj, name)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _scene_arrays(scene):
    # FP64 parameters; float32 inputs convert exactly
    verts = np.ascontiguousarray(_get(scene, "verts"), dtype=np.float64)
    sh = np.ascontiguousarray(_get(scene, "sh"), dtype=np.float64)
    opac = np.ascontiguousarray(_get(scene, "opacity"), dtype=np.float64)
    sig = np.ascontiguousarray(_get(scene, "sigma"), dtype=np.float64)
    deg = int(_get(scene, "sh_degree"))
    n = verts.shape[0]
    assert verts.shape == (n, 3, 3) and sh.shape == (n, (deg + 1) ** 2, 3)
    assert opac.shape == (n,) and sig.shape == (n,)
    return n, verts, sh, opac, sig, deg


def _cam_array(cam):
    a = np.zeros(21, dtype=np.float64)
    a[0:9] = np.asarray(_get(cam, "R"), dtype=np.float64).reshape(9)
    a[9:12] = np.asarray(_get(cam, "t"), dtype=np.float64).reshape(3)
    a[12] = _get(cam, "fx"); a[13] = _get(cam, "fy")
    a[14] = _get(cam, "cx"); a[15] = _get(cam, "cy")
    a[16] = _get(cam, "W"); a[17] = _get(cam, "H")
    a[18:21] = np.asarray(_get(cam, "bg"), dtype=np.float64).reshape(3)
    return a


def _const_array(consts):
    c = consts or DEFAULT_CONSTS
    return np.array([c["alpha_max"], c["alpha_min"], c["t_eps"], c["z_near"], c["r_min"],
                     c["tile"], c["rect_pad"], c.get("window", 0), c.get("sort", 0)], dtype=np.float64)


def render(scene, cam, consts=None, brute: bool = False, pix_mask=None, flags: bool = False,
           alt_capacity: int = 1 << 16):
    """Image [3,H,W], final transmittance [H,W], kept-fragment count [H,W] (FP64).

    With ``flags`` also returns the per-pixel ambiguity bits (AMB_*), the image error
    estimate, and ``alts``: for each pixel with a decision in the FP32 band, every
    outcome reached by taking such decisions either way (records of ALT_DTYPE: pixel
    index y * W + x, kept count, colour, T), at most ``alt_capacity`` records (pixels
    beyond carry AMB_UNRES)."""
    lib = _load()
    n, verts, sh, opac, sig, deg = _scene_arrays(scene)
    W, H = int(_get(cam, "W")), int(_get(cam, "H"))
    img = np.zeros((3, H, W), dtype=np.float64)
    T = np.ones((H, W), dtype=np.float64)
    nk = np.zeros((H, W), dtype=np.int32)
    fl = np.zeros((H, W), dtype=np.uint8) if flags else None
    err = np.zeros((H, W), dtype=np.float64) if flags else None
    pm = None if pix_mask is None else np.ascontiguousarray(pix_mask, dtype=np.uint8).reshape(H, W)
    if flags:
        alts = np.zeros(alt_capacity, dtype=ALT_DTYPE)
        n_alt = ctypes.c_size_t(0)
        rc = lib.orc_render_alts(n, _ptr(verts), _ptr(sh), deg, _ptr(opac), _ptr(sig), _ptr(_cam_array(cam)),
                                 _ptr(_const_array(consts)), int(bool(brute)), _ptr(pm), _ptr(img), _ptr(T),
                                 _ptr(nk), _ptr(fl), _ptr(err), _ptr(alts), alt_capacity, ctypes.byref(n_alt))
    else:
        rc = lib.orc_render(n, _ptr(verts), _ptr(sh), deg, _ptr(opac), _ptr(sig), _ptr(_cam_array(cam)),
                            _ptr(_const_array(consts)), int(bool(brute)), _ptr(pm), _ptr(img), _ptr(T),
                            _ptr(nk), None, None)
    if rc != 0:
        raise ValueError(f"orc_render failed ({rc})")
    out = dict(image=img, T_final=T, n_kept=nk)
    if flags:
        out.update(flags=fl, err=err, alts=alts[:min(n_alt.value, alt_capacity)].copy())
    return out


def render_stats(scene, cam, consts=None):
    """Pruning statistics per triangle (Sec. 3.3 "Pruning"): max_weight = largest T o
    over the triangle's composited fragments, n_pix = pixels where it was composited,
    amb = it took part in a pixel within the FP32 band."""
    lib = _load()
    n, verts, sh, opac, sig, deg = _scene_arrays(scene)
    mw = np.zeros(n, dtype=np.float64)
    npix = np.zeros(n, dtype=np.int32)
    amb = np.zeros(n, dtype=np.uint8)
    rc = lib.orc_render_stats(n, _ptr(verts), _ptr(sh), deg, _ptr(opac), _ptr(sig), _ptr(_cam_array(cam)),
                              _ptr(_const_array(consts)), _ptr(mw), _ptr(npix), _ptr(amb))
    if rc != 0:
        raise ValueError(f"orc_render_stats failed ({rc})")
    return dict(max_weight=mw, n_pix=npix, amb=amb)


def render_solid(scene, cam, consts=None, pix_mask=None):
    """Solid-triangle image [3,H,W], winning triangle id [H,W] (-1: background) and the
    per-pixel FP32-band flags: the sigma -> 0, o = 1 limit of the splat render. With
    pix_mask [H,W] only the pixels where it is non-zero are evaluated."""
    lib = _load()
    n, verts, sh, opac, sig, deg = _scene_arrays(scene)
    W, H = int(_get(cam, "W")), int(_get(cam, "H"))
    img = np.zeros((3, H, W), dtype=np.float64)
    ids = np.zeros((H, W), dtype=np.int32)
    fl = np.zeros((H, W), dtype=np.uint8)
    pm = None if pix_mask is None else np.ascontiguousarray(pix_mask, dtype=np.uint8).reshape(H, W)
    rc = lib.orc_render_solid(n, _ptr(verts), _ptr(sh), deg, _ptr(opac), _ptr(sig), _ptr(_cam_array(cam)),
                              _ptr(_const_array(consts)), _ptr(pm), _ptr(img), _ptr(ids), _ptr(fl))
    if rc != 0:
        raise ValueError(f"orc_render_solid failed ({rc})")
    return dict(image=img, id=ids, flags=fl)


def render_grad(scene, cam, dL_dimage, consts=None, pix_mask=None, tri_mask=None):
    """Parameter gradients of sum(dL_dimage * image) in FP64."""
    lib = _load()
    n, verts, sh, opac, sig, deg = _scene_arrays(scene)
    W, H = int(_get(cam, "W")), int(_get(cam, "H"))
    g = np.ascontiguousarray(dL_dimage, dtype=np.float64).reshape(3, H, W)
    K = (deg + 1) ** 2
    dv = np.zeros((n, 3, 3)); dsh = np.zeros((n, K, 3)); do = np.zeros(n); ds = np.zeros(n)
    pm = None if pix_mask is None else np.ascontiguousarray(pix_mask, dtype=np.uint8).reshape(H, W)
    tm = None if tri_mask is None else np.ascontiguousarray(tri_mask, dtype=np.uint8).reshape(n)
    rc = lib.orc_render_grad(n, _ptr(verts), _ptr(sh), deg, _ptr(opac), _ptr(sig),
                             _ptr(_cam_array(cam)), _ptr(_const_array(consts)), _ptr(g), _ptr(pm),
                             _ptr(tm), _ptr(dv), _ptr(dsh), _ptr(do), _ptr(ds))
    if rc != 0:
        raise ValueError(f"orc_render_grad failed ({rc})")
    return dict(verts=dv, sh=dsh, opacity=do, sigma=ds)


def tri_info(scene, cam, consts=None):
    """Per-triangle FP64 quantities: projected vertices, depth, incenter, inradius,
    shrink factor, tight rectangle, pixel / tile rectangles, colour and flags."""
    lib = _load()
    n, verts, sh, opac, sig, deg = _scene_arrays(scene)
    f = np.zeros((max(n, 1), 24)); i = np.zeros((max(n, 1), 12), dtype=np.int32)
    rc = lib.orc_tri_info(n, _ptr(verts), _ptr(sh), deg, _ptr(opac), _ptr(sig),
                          _ptr(_cam_array(cam)), _ptr(_const_array(consts)), _ptr(f), _ptr(i))
    if rc != 0:
        raise ValueError(f"orc_tri_info failed ({rc})")
    f = f[:n]; i = i[:n]
    return dict(q=f[:, 0:6].reshape(n, 3, 2), z=f[:, 6:9], depth=f[:, 9], s=f[:, 10:12],
                r=f[:, 12], f=f[:, 13], rect=f[:, 14:18], rgb=f[:, 18:21], dir=f[:, 21:24],
                cull=i[:, 0], rect_state=i[:, 1], pix=i[:, 2:6], tiles=i[:, 6:10],
                amb=i[:, 10], ntiles=i[:, 11])


def tile_pairs(scene, cam, consts=None, info=None):
    """(tile id, triangle id) pairs ordered by (tile, FP64 depth, id), from the FP64
    tight rectangles (Supp. "Tile assignment", "Depth sorting")."""
    info = info if info is not None else tri_info(scene, cam, consts)
    tile = int((consts or DEFAULT_CONSTS)["tile"])
    tx = (int(_get(cam, "W")) + tile - 1) // tile
    tiles, ids, depth = [], [], []
    for t in np.nonzero(info["ntiles"] > 0)[0]:
        x0, y0, x1, y1 = info["tiles"][t]
        ty, txx = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
        tt = (ty * tx + txx).reshape(-1)
        tiles.append(tt); ids.append(np.full(tt.size, t)); depth.append(np.full(tt.size, info["depth"][t]))
    if not tiles:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    tiles = np.concatenate(tiles); ids = np.concatenate(ids); depth = np.concatenate(depth)
    order = np.lexsort((ids, depth, tiles))
    return tiles[order].astype(np.int64), ids[order].astype(np.int64)


def tri2d(q):
    """Outward unit normals n [3,2], offsets d [3], incenter s [2], inradius r, sides ell [3]."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(6)
    out = np.zeros(15)
    lib.orc_tri2d(_ptr(q), _ptr(out))
    return dict(n=out[0:6].reshape(3, 2), d=out[6:9], s=out[9:11], r=out[11], ell=out[12:15])


def window(q, sigma, pts):
    """ratio = phi(p)/phi(s) and I = ReLU(ratio)^sigma at points [M,2]."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(6)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    ratio = np.zeros(len(pts)); I = np.zeros(len(pts))
    lib.orc_window(_ptr(q), float(sigma), len(pts), _ptr(pts), _ptr(ratio), _ptr(I))
    return ratio, I


def window_sigmoid(q, sigma, pts):
    """Eq. indicator2: signed distance phi(p) (pixels) and I = sigmoid(-phi / sigma)."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(6)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    phi = np.zeros(len(pts)); I = np.zeros(len(pts))
    lib.orc_window_sigmoid(_ptr(q), float(sigma), len(pts), _ptr(pts), _ptr(phi), _ptr(I))
    return phi, I


def sh_eval(deg, dirs):
    """Real SH basis values [M, (deg+1)^2] at unit directions [M,3]."""
    lib = _load()
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(dirs), (deg + 1) ** 2))
    rc = lib.orc_sh_eval(int(deg), len(dirs), _ptr(dirs), _ptr(out))
    if rc != 0:
        raise ValueError("bad degree")
    return out


def prune_keep(max_weight, n_pix, tau_prune: float, min_views: int = 2, min_pixels: int = 2):
    """The pruning rule of Sec. 3.3 ("Pruning") over per-view statistics max_weight
    [V, N] (largest blending weight T o of each triangle in each view) and n_pix [V, N]
    (pixels where it was composited): a triangle is kept when its largest weight over
    all views reaches tau_prune and it was rendered with more than one pixel
    (n_pix >= min_pixels) in at least min_views views ("at least twice")."""
    mw = np.asarray(max_weight, dtype=np.float64)
    npx = np.asarray(n_pix)
    keep = np.zeros(mw.shape[1], dtype=bool)
    for i in range(mw.shape[1]):
        best = max(mw[v, i] for v in range(mw.shape[0]))
        views = sum(1 for v in range(mw.shape[0]) if npx[v, i] >= min_pixels)
        keep[i] = best >= tau_prune and views >= min_views
    return keep
