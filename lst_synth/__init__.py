"""Seeded synthetic inputs (detector description, events, pixel seeds) for the LST hot path.

Shared by the CPU oracle tests, the CUDA library tests and the benchmark.  It simulates
detector data only and contains none of the tracking method's arithmetic.
"""
from .geometry import Geometry, MODULE_DTYPE, PT_PER_CM  # noqa: F401
from .events import Event, PLS_DTYPE, TRACK_DTYPE, event_from_tracks, random_tracks  # noqa: F401
from .workloads import make_event, workload_geometry, geometry, seed_of  # noqa: F401
