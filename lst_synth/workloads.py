"""The five synthetic workloads (seeded) that stand in for the paper's CMS ttbar PU200 sample.

Seeds: workload c, event i -> ``1_000_003 * c + i``; the tiny workload is fixed at seed 0.

  tiny        barrel only, 10 tracks, pT U[1,10] GeV, |eta| < 1, z0 ~ N(0, 5 cm), no noise
  pu200       barrel + 10 disks, 4000 tracks, pT pdf ~ 1/pT^2 above 0.5 GeV (capped at 200),
              |eta| < 2.4, + 20 % noise hits; optional pixel seeds (recipe of highocc)
  batched     64 barrel-only events with U{500..6000} tracks, each generated like ``tiny``
  serving     barrel + disks, U{2000..8000} tracks, pu200 generator with 20 % noise
  highocc     12000 tracks + 30 % noise + pixel seeds (1 % pT, 1 mrad phi smear, 10 % fakes),
              16 events per batch
"""
from __future__ import annotations

import numpy as np

from . import events as E
from . import geometry as G

SEED_STRIDE = 1_000_003
WORKLOAD_ID = {"tiny": 1, "pu200": 2, "batched": 3, "serving": 4, "highocc": 5}

_GEOMS: dict = {}


def geometry(barrel_only: bool, realistic: bool = False, endcap_2s: bool = False) -> G.Geometry:
    """The detector of a workload; ``realistic`` tilts the inner-barrel rows and
    ``endcap_2s`` makes the outer endcap rings 2S (features of the paper's Fig. 1)."""
    key = (barrel_only, realistic, endcap_2s)
    if key not in _GEOMS:
        _GEOMS[key] = G.Geometry(barrel_only=barrel_only, realistic=realistic, endcap_2s=endcap_2s)
    return _GEOMS[key]


def seed_of(workload: str, i: int) -> int:
    if workload == "tiny":
        return 0
    return SEED_STRIDE * WORKLOAD_ID[workload] + i


def make_event(workload: str, i: int = 0, *, n_tracks=None, with_pls=None, exact=False,
               realistic=False, triplet_frac=0.0, endcap_2s=False) -> E.Event:
    """Event ``i`` of ``workload`` (``n_tracks``/``with_pls`` override the recipe;
    ``realistic`` simulates it in the geometry with tilted inner-barrel modules;
    ``endcap_2s`` in the geometry whose outer endcap rings are 2S modules;
    ``triplet_frac`` of the pixel seeds are triplets, three hits instead of four)."""
    seed = seed_of(workload, i)
    rng = np.random.default_rng(seed + 7)
    if workload in ("tiny", "batched"):
        geom = geometry(True, realistic)
        n = n_tracks if n_tracks is not None else (10 if workload == "tiny" else int(rng.integers(500, 6001)))
        t = E.random_tracks(rng, n, pt_mode="uniform", pt_lo=1.0, pt_hi=10.0, eta_max=1.0)
        return E.event_from_tracks(geom, t, seed, noise_frac=0.0, exact=exact,
                                   with_pls=bool(with_pls), triplet_frac=triplet_frac)
    geom = geometry(False, realistic, endcap_2s)
    if workload == "pu200":
        n, noise, pls = 4000, 0.20, False
    elif workload == "serving":
        n, noise, pls = int(rng.integers(2000, 8001)), 0.20, False
    elif workload == "highocc":
        n, noise, pls = 12000, 0.30, True
    else:
        raise ValueError(workload)
    if n_tracks is not None:
        n = n_tracks
    if with_pls is not None:
        pls = with_pls
    t = E.random_tracks(rng, n, pt_mode="inv2", pt_lo=0.5, eta_max=2.4)
    return E.event_from_tracks(geom, t, seed, noise_frac=0.0 if exact else noise, exact=exact,
                               with_pls=pls, triplet_frac=triplet_frac)


def workload_geometry(workload: str, realistic: bool = False) -> G.Geometry:
    return geometry(workload in ("tiny", "batched"), realistic)
