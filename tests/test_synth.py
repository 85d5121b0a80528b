"""Pins of the synthetic input generator (geometry, helices, resolution model)."""
import numpy as np

import lst_synth as S
from lst_synth import events as E
from lst_synth import geometry as G


def test_module_counts(barrel_geom, full_geom):
    # 24 z bins x ceil(2 pi r / 10) sectors on 6 layers; 10 disks x 9 rings
    assert barrel_geom.n_modules == 24 * (15 + 23 + 33 + 43 + 55 + 70) == 5736
    assert full_geom.n_modules == 5736 + 10 * (16 + 22 + 29 + 35 + 41 + 48 + 54 + 60 + 66)


def test_sector_edges_shared(full_geom):
    m = full_geom.modules
    # edge k+1 of a sector is bit-identical to edge k of the next sector (wrap included)
    for sub in (0, 1):
        sel = np.nonzero((m["subdet"] == sub) & (m["iphi"] == 0))[0][:20]
        for i0 in sel:
            n = int(m["nphi"][i0])
            row = m[i0:i0 + n]
            assert np.array_equal(row["e1x"][:-1], row["e0x"][1:])
            assert row["e1x"][-1] == row["e0x"][0] and row["e1y"][-1] == row["e0y"][0]


def test_exact_points_on_helix_circle(full_geom):
    rng = np.random.default_rng(1)
    t = E.random_tracks(rng, 200, pt_mode="inv2", pt_lo=0.5, eta_max=2.4)
    ev = E.event_from_tracks(full_geom, t, 3, exact=True, shuffle=False)
    R = t["pt"][ev.sim] / S.PT_PER_CM
    q = t["q"][ev.sim]
    cx = t["vx"][ev.sim] + q * R * np.sin(t["phi0"][ev.sim])
    cy = t["vy"][ev.sim] - q * R * np.cos(t["phi0"][ev.sim])
    d = np.hypot(ev.x.astype(np.float64) - cx, ev.y.astype(np.float64) - cy)
    # float32 rounding of coordinates up to ~270 cm
    assert np.max(np.abs(d - R)) < 2e-4 * np.maximum(1, np.max(np.abs([ev.x, ev.y])) / 100)
    # z grows linearly with turning angle
    assert ev.n_hits > 1000


def test_hits_inside_their_modules(full_geom):
    ev = S.make_event("pu200", 0)
    m = full_geom.modules[ev.det >> 1]
    up = (ev.det & 1).astype(np.float64)
    barrel = m["subdet"] == 0
    r = np.hypot(ev.x, ev.y)
    surf = m["surf"] + up * m["gap"] * np.where(barrel, 1.0, m["side"])
    # barrel: radius is the sensor radius; endcap: z is the sensor plane
    assert np.all(np.abs(r[barrel] - surf[barrel]) < 1e-3)
    assert np.all(np.abs(ev.z[~barrel] - surf[~barrel]) < 1e-4)
    ext = np.where(barrel, ev.z, r)
    assert np.all(ext > m["emin"] - 0.5) and np.all(ext < m["emax"] + 0.5)


def test_deterministic():
    a = S.make_event("serving", 3)
    b = S.make_event("serving", 3)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.det, b.det)
    c = S.make_event("serving", 4)
    assert c.n_hits != a.n_hits or not np.array_equal(a.x, c.x)


def test_workload_shapes():
    t = S.make_event("tiny")
    assert len(t.tracks) == 10 and t.n_hits < 150 and np.all(t.sim >= 0)
    p = S.make_event("pu200", 0, with_pls=True)
    noise = np.mean(p.sim < 0)
    assert 0.15 < noise < 0.18  # 20 % of the track hits
    real = p.pls_sim >= 0
    assert np.all(p.tracks["pt"][p.pls_sim[real]] >= 0.8)
    assert abs((~real).sum() / real.sum() - 0.10) < 0.01
