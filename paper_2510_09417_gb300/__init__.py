"""GB300-native level-synchronous planar Quickhull (VQhull, arxiv 2510.09417).

The hull path runs in the CUDA library libvqhull.so (sm_103a kernels behind
the C ABI of include/vqhull.h); this package builds it in-tree and binds it.
"""
from .libbuild import build  # noqa: F401
from .vqhull import (  # noqa: F401
    SYMBOLS, Config, Server, VQError, library_path, load, status_string, vq_get_config,
    vq_autotune, vq_debug_orient_f32, vq_debug_round_f32, vq_hull2d, vq_hull2d_aos, vq_hull2d_batched, vq_hull2d_host, vq_hull2d_noalloc, vq_last_stats, vq_profile_read,
    vq_set_config,
    vq_status_string, vq_version,
)
