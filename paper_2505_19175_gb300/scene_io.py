"""Scene checkpoints: the parameters of a triangle soup as one ``.npz`` file (vertices
[N,3,3], SH [N,(d+1)^2,3], opacity [N], sigma [N], SH degree; 59 floats per triangle at
degree 3, the count of Sec. 4)."""
from __future__ import annotations

import numpy as np

from .synth import Scene


def save(path: str, scene) -> None:
    """Write ``scene`` (a ``synth.Scene`` or ``renderer.SceneTensors``) to ``path``."""
    def host(x):
        return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    np.savez(path, verts=host(scene.verts).astype(np.float32), sh=host(scene.sh).astype(np.float32),
             opacity=host(scene.opacity).astype(np.float32), sigma=host(scene.sigma).astype(np.float32),
             sh_degree=np.int32(scene.sh_degree))


def load(path: str) -> Scene:
    with np.load(path) as z:
        n = z["verts"].shape[0]
        deg = int(z["sh_degree"])
        verts, sh = z["verts"].reshape(n, 3, 3), z["sh"].reshape(n, (deg + 1) ** 2, 3)
        if z["opacity"].shape != (n,) or z["sigma"].shape != (n,):
            raise ValueError(f"{path}: inconsistent array shapes")
        return Scene(verts.copy(), sh.copy(), z["opacity"].copy(), z["sigma"].copy(), deg)
