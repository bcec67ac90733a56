"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the bench.

This package holds workload definitions and random-number recipes only: it
draws hits, truth tracks and multistart seeds, and it computes none of the
retina response, its derivatives, the search or the deduplication.
"""
from .events import (  # noqa: F401
    MODEL_TOY2D,
    MODEL_VELO_SLOPES,
    Event,
    Batch,
    Workload,
    WORKLOADS,
    VELO_PLANES_Z,
    SVELO_PLANES_Z,
    make_svelo_event,
    slopes_to_angles,
    make_toy2d_event,
    make_velo_event,
    make_event,
    make_batch,
    batch_of,
    uniform_seeds,
    seednet_init_params,
    close_tracks_event,
)
