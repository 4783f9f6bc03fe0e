"""Helpers shared by the GPU parity tests (run the CUDA path through the C ABI and
rebuild the expected tile lists from its own unsorted per-item outputs)."""
import numpy as np


def gpu_forward(scene, cams, sync_pairs=True):
    import torch
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    ctx.preprocess(st, cams)
    ctx.bin_sort(sync=sync_pairs)
    imgs = new_images(cams)
    T = [torch.empty((c.H, c.W), device="cuda") for c in cams]
    nc = [torch.empty((c.H, c.W), device="cuda", dtype=torch.int32) for c in cams]
    ctx.render_fwd(imgs, T, nc)
    ctx.check()
    torch.cuda.synchronize()
    return ([x.cpu().numpy().astype(np.float64) for x in imgs], [x.cpu().numpy().astype(np.float64) for x in T],
            [x.cpu().numpy() for x in nc], ctx, st)


def gpu_backward(ctx, st, dls):
    import torch
    ctx.render_bwd([torch.as_tensor(np.ascontiguousarray(d, np.float32)).cuda() for d in dls])
    dv = torch.empty_like(st.verts)
    dsh = torch.empty_like(st.sh)
    do = torch.empty_like(st.opacity)
    ds = torch.empty_like(st.sigma)
    ctx.preprocess_bwd(dv, dsh, do, ds)
    ctx.check()
    torch.cuda.synchronize()
    return dict(verts=dv.cpu().numpy().astype(np.float64), sh=dsh.cpu().numpy().astype(np.float64),
                opacity=do.cpu().numpy().astype(np.float64), sigma=ds.cpu().numpy().astype(np.float64))


def expected_pairs_from_items(ctx, cams):
    """Stable sort, by 64-bit key (global tile << 32 | depth bits), of the pairs emitted
    in item order from the GPU's own per-item rectangles and depth keys."""
    rects = ctx.debug("rects").astype(np.int64) // 16     # pixel rectangle -> tile rectangle
    nt = ctx.debug("ntiles").astype(np.int64)
    dk = ctx.debug("depth_keys").astype(np.uint64)
    n_items = len(nt)
    n = n_items // len(cams)
    tile_base, tx_of = [], []
    tb = 0
    for c in cams:
        tx = (c.W + 15) // 16
        ty = (c.H + 15) // 16
        tile_base.append(tb)
        tx_of.append(tx)
        tb += tx * ty
    keys, vals = [], []
    for m in np.nonzero(nt > 0)[0]:
        v = m // n
        x0, y0, x1, y1 = rects[m]
        ty, txx = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
        t = (tile_base[v] + ty * tx_of[v] + txx).reshape(-1).astype(np.uint64)
        assert len(t) == nt[m]
        keys.append((t << np.uint64(32)) | dk[m])
        vals.append(np.full(len(t), m, np.uint64))
    if not keys:
        return np.zeros(0, np.uint64), np.zeros(0, np.uint64)
    keys = np.concatenate(keys)
    vals = np.concatenate(vals)
    order = np.argsort(keys, kind="stable")
    return (keys[order] >> np.uint64(32)), vals[order]


def flagged_fraction(flags):
    return float(np.mean(flags != 0))


IMAGE_TOL = 1e-4          # absolute, per channel, and for the final transmittance
UNRESOLVED_CAP = 1e-4     # at most 0.01 % of the checked pixels without listed outcomes


def check_image(img, T, ref, sel=None, label="", n_kept=None, tol=IMAGE_TOL):
    """Every checked pixel of a GPU image against the FP64 oracle (``ref`` from
    ``O.render(..., flags=True)``), with no pixel left out:
    - a pixel whose decisions FP32 resolves: colour and T within ``tol``;
    - a pixel with a decision in the FP32 band (alpha vs 1/255, the T stop, two depths):
      equal, within ``tol`` plus the oracle's error estimate, to one of the outcomes the
      oracle lists for it (each ambiguous decision taken either way);
    - a pixel whose only flag is its error estimate (a steep window): within ``tol``
      plus that estimate;
    - pixels whose outcomes were not all listed count against a cap of 0.01 %.
    ``sel`` (bool [H,W]) limits the check to sampled pixels; with ``T`` None only the
    colour is compared (a caller without the final transmittance). Prints the flagged
    counts.
    Returns the mask of pixels checked at ``tol`` alone (FP32-resolved, gradient-
    resolved), for building a loss on them."""
    import oracle as O
    fl = ref["flags"]
    H, W = fl.shape
    sel = np.ones((H, W), bool) if sel is None else np.asarray(sel, bool)
    img_flags = fl & np.uint8(0xFF ^ O.AMB_GRAD)
    clean = sel & (img_flags == 0)
    dec = sel & ((fl & O.AMB_DECISION) != 0) & ((fl & O.AMB_UNRES) == 0)
    sens = sel & (img_flags == O.AMB_SENS)
    unres = sel & ((fl & O.AMB_UNRES) != 0)
    n = int(sel.sum())
    print(f"[flagged] {label}: {int((sel & (img_flags != 0)).sum())} of {n} pixels "
          f"({(sel & (img_flags != 0)).sum() / max(n, 1):.4%}; decision {int(dec.sum())}, estimate-only "
          f"{int(sens.sum())}, unresolved {int(unres.sum())}); gradient-only {int((sel & (fl == O.AMB_GRAD)).sum())}")
    err = np.abs(img - ref["image"])[:, clean]
    assert err.size == 0 or err.max() <= tol, f"{label}: image max err {err.max():.3e} on resolved pixels"
    if T is not None:
        terr = np.abs(T - ref["T_final"])[clean]
        assert terr.size == 0 or terr.max() <= tol, f"{label}: T max err {terr.max():.3e} on resolved pixels"
    if n_kept is not None:
        np.testing.assert_array_equal(n_kept[clean], ref["n_kept"][clean])
    est = ref["err"]
    if sens.any():
        e = np.abs(img - ref["image"])[:, sens].max(0)
        et = np.abs(T - ref["T_final"])[sens] if T is not None else 0.0
        bound = tol + est[sens]
        assert np.all(e <= bound) and np.all(et <= bound), f"{label}: estimate-only pixel beyond tol + estimate"
    if dec.any():
        alts = ref["alts"]
        ys, xs = np.nonzero(dec)
        for y, x in zip(ys, xs):
            a = alts[alts["pix"] == y * W + x]
            assert len(a) > 0, f"{label}: no outcome listed for flagged pixel ({x}, {y})"
            d = np.abs(a["image"] - img[:, y, x][None]).max(1)
            if T is not None:
                d = np.maximum(d, np.abs(a["T"] - T[y, x]))
            ok = d <= tol + est[y, x]
            if n_kept is not None:
                ok &= a["n_kept"] == n_kept[y, x]
            assert ok.any(), (f"{label}: pixel ({x}, {y}) matches none of its {len(a)} outcomes "
                              f"(nearest {d.min():.3e}, estimate {est[y, x]:.2e})")
    assert unres.sum() <= UNRESOLVED_CAP * n, f"{label}: {int(unres.sum())} unresolved pixels of {n}"
    return sel & (fl == 0)


def loss_pixels(ref, sel=None):
    """Pixels that take part in a gradient comparison: every decision, the image value
    and the gradient contribution resolved in FP32 (flags == 0), within ``sel``."""
    ok = ref["flags"] == 0
    return ok if sel is None else ok & np.asarray(sel, bool)
