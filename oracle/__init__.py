"""FP64 CPU oracle for the triangle-splat rasterizer (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package. The product path never does.
"""
from .oracle import (  # noqa: F401
    DEFAULT_CONSTS, EXACT_CONSTS, build, render, render_grad, render_stats, render_solid, tri_info, tri2d,
    window, window_sigmoid, sh_eval, tile_pairs, prune_keep, set_threads, max_threads, WINDOW_POWER, WINDOW_SIGMOID,
    SORT_TILE, SORT_PIXEL,
    AMB_SKIP, AMB_STOP, AMB_ORDER, AMB_SENS, AMB_CULL, AMB_UNRES, AMB_GRAD, AMB_DECISION, ALT_DTYPE,
)
