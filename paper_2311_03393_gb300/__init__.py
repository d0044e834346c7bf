"""GB300-native sketched discord mining (Yeh et al., arXiv 2311.03393).

The computation lives in libtsketch.so (CUDA, sm_103a) behind the C ABI of
include/tsketch.h; this package is its thin Python binding plus seeded
synthetic workloads (synth).
"""
from .api import (  # noqa: F401
    ab_discords,
    DiscordScores,
    context,
    default_excl,
    dimension_detection,
    discord_topk,
    exact_discords,
    launch_count,
    mp_abjoin,
    mp_backward,
    mp_selfjoin,
    mp_selfjoin_update,
    pack_batch,
    profile_enable,
    profile_read,
    refine_dimensions,
    reserve,
    set_tile_rows,
    sketched_discords,
    sync,
    ts_sketch_build,
    ts_sketch_point_update,
    ts_sketch_update_dims,
)
