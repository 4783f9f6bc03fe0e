"""FP64 reference of the densification moves and the size regulariser (Sec. 3.3
"Densification"; Sec. 3.4 "Optimization", L_s). TEST INFRASTRUCTURE ONLY (see the
package docstring).

Readings of the paper, shared with the CUDA path's contract:
  * midpoint subdivision replaces a selected triangle (v0, v1, v2) by the four
    triangles of its edge midpoints m01, m12, m02: (v0, m01, m02) in place, then
    (m01, v1, m12), (m02, m12, v2), (m01, m12, m02) appended; colour, opacity and
    sigma are copied (the children tile the parent, so no opacity change);
  * a selected triangle with area below tau_small is cloned instead: the clone is
    the triangle translated by noise_scale (a e1 + b e2), e1 = (v1 - v0) / |v1 - v0|,
    e2 = n x e1 with n the unit normal, (a, b) the caller's standard normal draws;
    both copies take opacity 1 - sqrt(1 - o), so that the two overlapping copies
    composite to the original opacity (the probability-preserving move of MCMC
    densification);
  * appended triangles follow the order of the selection list;
  * L_s = 2 / |(v1 - v0) x (v2 - v0)| per triangle, summed with a caller weight
    (weight = beta / n gives the mean); below |cross| = 1e-12 the term and its
    gradient are 0.
"""
from __future__ import annotations

import numpy as np

EPS_CROSS = 1e-12


def _f64(x):
    return np.asarray(x, dtype=np.float64)


def area(verts):
    v = _f64(verts)
    return 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)


def subdivide(verts, sh, opacity, sigma, sel, noise, noise_scale: float, tau_small: float):
    """Returns (verts, sh, opacity, sigma) of the densified scene (FP64)."""
    v = _f64(verts).copy()
    sh = _f64(sh).copy()
    o = _f64(opacity).copy()
    s = _f64(sigma).copy()
    noise = _f64(noise).reshape(-1, 2)
    add_v, add_sh, add_o, add_s = [], [], [], []
    for k, i in enumerate(np.asarray(sel, dtype=np.int64)):
        v0, v1, v2 = v[i].copy()
        cross = np.cross(v1 - v0, v2 - v0)
        if 0.5 * np.linalg.norm(cross) >= tau_small:
            m01, m12, m02 = (v0 + v1) / 2, (v1 + v2) / 2, (v0 + v2) / 2
            v[i] = (v0, m01, m02)
            for tri in ((m01, v1, m12), (m02, m12, v2), (m01, m12, m02)):
                add_v.append(np.array(tri)); add_sh.append(sh[i]); add_o.append(o[i]); add_s.append(s[i])
        else:
            nrm = cross / max(np.linalg.norm(cross), EPS_CROSS)
            e1 = (v1 - v0) / max(np.linalg.norm(v1 - v0), EPS_CROSS)
            e2 = np.cross(nrm, e1)
            t = noise_scale * (noise[k, 0] * e1 + noise[k, 1] * e2)
            o[i] = 1.0 - np.sqrt(1.0 - o[i])
            add_v.append(v[i] + t[None]); add_sh.append(sh[i]); add_o.append(o[i]); add_s.append(s[i])
    if add_v:
        v = np.concatenate([v, np.stack(add_v)])
        sh = np.concatenate([sh, np.stack(add_sh)])
        o = np.concatenate([o, np.array(add_o)])
        s = np.concatenate([s, np.array(add_s)])
    return v, sh, o, s


def size_reg(verts, weight: float = 1.0):
    """(weight * sum_i 2 / |c_i|, d/dverts [N,3,3]) with c_i = (v1 - v0) x (v2 - v0)."""
    v = _f64(verts)
    e1, e2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    c = np.cross(e1, e2)
    nc = np.linalg.norm(c, axis=1)
    ok = nc >= EPS_CROSS
    L = np.where(ok, 2.0 / np.where(ok, nc, 1.0), 0.0)
    g = np.where(ok[:, None], -2.0 * c / np.where(ok, nc, 1.0)[:, None] ** 3, 0.0)   # dL/dc
    d1 = np.cross(e2, g)            # dL/dv1 = e2 x g
    d2 = np.cross(g, e1)            # dL/dv2 = g x e1
    grad = np.stack([-(d1 + d2), d1, d2], axis=1)
    return weight * L.sum(), weight * grad
