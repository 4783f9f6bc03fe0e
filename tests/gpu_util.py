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
