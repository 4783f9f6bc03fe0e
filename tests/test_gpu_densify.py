"""Densification moves and the size regulariser on the GPU against the FP64 reference
(Sec. 3.3, Sec. 3.4): vertex positions within FP32 rounding, attributes exactly, the
same subdivide / clone decisions, and L_s with its gradient."""
import numpy as np
import pytest

from oracle import densify as D

pytestmark = pytest.mark.gpu


def _scene(n, seed, deg=2):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-2, 2, (n, 3))
    scale = np.exp(rng.uniform(np.log(0.01), np.log(0.5), n))
    v = c[:, None, :] + scale[:, None, None] * rng.standard_normal((n, 3, 3))
    sh = rng.standard_normal((n, (deg + 1) ** 2, 3))
    return (v.astype(np.float32), sh.astype(np.float32), rng.uniform(0.05, 0.95, n).astype(np.float32),
            rng.uniform(0.3, 3.0, n).astype(np.float32))


@pytest.mark.parametrize("n,k", [(1000, 300), (5000, 2500), (700, 1)])
def test_densify_matches_reference(n, k):
    import torch
    from paper_2505_19175_gb300.densify import densify
    from paper_2505_19175_gb300.renderer import Context
    v, sh, o, s = _scene(n, seed=n + k)
    rng = np.random.default_rng(k)
    sel = rng.choice(n, k, replace=False).astype(np.int32)
    noise = rng.standard_normal((k, 2)).astype(np.float32)
    areas = D.area(v[sel])
    tau = float(np.median(areas))
    keep = np.abs(areas - tau) > 1e-4 * tau          # decisions away from the FP32 band
    sel, noise = sel[keep], noise[keep]
    k = len(sel)
    cap = n + 3 * k + 5
    T = lambda a, shape: torch.as_tensor(np.concatenate([a, np.zeros(shape, a.dtype)])).cuda().contiguous()
    tv, tsh = T(v, (cap - n, 3, 3)), T(sh, (cap - n,) + sh.shape[1:])
    to, ts = T(o, (cap - n,)), T(s, (cap - n,))
    n_new = densify(Context(), tv, tsh, to, ts, n, torch.as_tensor(sel).cuda(), torch.as_tensor(noise).cuda(),
                    0.03, tau, sh_degree=2)
    rv, rsh, ro, rs = D.subdivide(v, sh, o, s, sel, noise, 0.03, tau)
    assert n_new == len(rv)
    np.testing.assert_allclose(tv[:n_new].cpu().numpy(), rv, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(tsh[:n_new].cpu().numpy(), rsh.astype(np.float32))
    np.testing.assert_allclose(to[:n_new].cpu().numpy(), ro, rtol=2e-6)
    np.testing.assert_array_equal(ts[:n_new].cpu().numpy(), rs.astype(np.float32))


def test_densify_rejects_small_capacity_and_bad_indices():
    import torch
    from paper_2505_19175_gb300.densify import densify
    from paper_2505_19175_gb300.native import TriError
    from paper_2505_19175_gb300.renderer import Context
    v, sh, o, s = _scene(50, 7)
    t = [torch.as_tensor(x).cuda() for x in (v, sh, o, s)]
    sel = torch.arange(10, dtype=torch.int32, device="cuda")
    noise = torch.zeros((10, 2), device="cuda")
    with pytest.raises(TriError):
        densify(Context(), *t, 50, sel, noise, 0.1, 0.0, sh_degree=2)     # capacity 50 < 80
    cap = 50 + 30
    T = lambda a, shape: torch.as_tensor(np.concatenate([a, np.zeros(shape, a.dtype)])).cuda()
    tt = [T(v, (30, 3, 3)), T(sh, (30, 9, 3)), T(o, (30,)), T(s, (30,))]
    ctx = Context()
    bad = torch.tensor([3, 99], dtype=torch.int32, device="cuda")           # 99 is out of range
    n_new = densify(ctx, *tt, 50, bad, torch.zeros((2, 2), device="cuda"), 0.1, 0.0, sh_degree=2)
    assert n_new == 53
    assert cap >= n_new


def test_size_regulariser_matches_reference():
    import torch
    from paper_2505_19175_gb300.densify import size_reg
    v, _, _, _ = _scene(20000, 8)
    tv = torch.as_tensor(v).cuda()
    grad = torch.zeros_like(tv)
    loss = size_reg(tv, weight=0.25, grad=grad)
    rl, rg = D.size_reg(v, 0.25)
    np.testing.assert_allclose(float(loss), rl, rtol=1e-4)
    g = grad.cpu().numpy()
    np.testing.assert_allclose(g, rg, rtol=1e-4, atol=1e-4 * np.abs(rg).max())
