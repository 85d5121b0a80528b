"""Single noiseless helix events and hit edits, for the oracle's rejection-side pins.

Every case starts from points the input generator puts exactly on a helix (float64
geometry rounded once to float32), then moves one doublet or one seed parameter by an
amount chosen from the geometry of the reading, in float64 here, so that a cut's decision
is set by the construction and not by the oracle's own arithmetic.
"""
from __future__ import annotations

import numpy as np

import lst_synth as S
from lst_synth import events as E

RMIN = 0.8 / S.PT_PER_CM          # curvature radius of the 0.8 GeV threshold (Sec. 1), cm
EDIR = 3.0 * np.sqrt(2.0) * 0.003  # 3 sigma of a two-hit r-phi difference (30 um each), cm


def track(pt, phi0, eta, q=1, v=(0.0, 0.0, 0.0)):
    t = np.zeros(1, E.TRACK_DTYPE)
    t["pt"], t["phi0"], t["eta"], t["q"] = pt, phi0, eta, q
    t["vx"], t["vy"], t["vz"] = v
    return t


def event(geom, t, pls=False):
    """Hits of track(s) ``t`` in crossing order (no shuffle), exact points, exact seeds."""
    return E.event_from_tracks(geom, t, 5, exact=True, with_pls=pls, fake_pls_frac=0.0, shuffle=False)


def doublets(ev):
    """[(module, lower hit, upper hit)] of the modules where both sensor hits of the first
    track landed on the same module, in crossing order."""
    mod = (ev.det >> 1).astype(np.int64)
    sen = ev.det & 1
    out = []
    i = 0
    while i + 1 < ev.n_hits:
        if ev.sim[i] == ev.sim[i + 1] and mod[i] == mod[i + 1] and sen[i] == 0 and sen[i + 1] == 1:
            out.append((int(mod[i]), i, i + 1))
            i += 2
        else:
            i += 1
    return out


def clean_track(geom, pt, eta, n_layers, q=1, v=(0.0, 0.0, 0.0), pls=False, phis=None, vz=None):
    """The first azimuth in ``phis`` whose track gives ``n_layers`` clean doublets."""
    for phi0 in (phis if phis is not None else np.linspace(0.11, 6.1, 41)):
        vv = v if vz is None else (v[0], v[1], vz)
        t = track(pt, phi0, eta, q, vv)
        ev = event(geom, t, pls)
        d = doublets(ev)
        if len(d) == n_layers:
            return t, ev, d
    raise AssertionError("no clean track found")


def points(ev):
    return np.stack([ev.x, ev.y, ev.z], 1).astype(np.float64)


def edited(ev, changes: dict, pls=None):
    """Copy of ``ev`` with hits moved: changes = {hit index: (x, y, z)} (float64)."""
    x, y, z = ev.x.copy(), ev.y.copy(), ev.z.copy()
    for i, p in changes.items():
        x[i], y[i], z[i] = np.float32(p[0]), np.float32(p[1]), np.float32(p[2])
    return E.Event(x, y, z, ev.det.copy(), ev.sim.copy(), ev.tracks,
                   ev.pls.copy() if pls is None else pls, ev.pls_sim.copy())


def outward(t, p):
    """Unit transverse vector from the helix axis through point p (the convex side)."""
    _, _, cx, cy = E.helix_centre(t)
    d = np.array([p[0] - cx[0], p[1] - cy[0]])
    return d / np.linalg.norm(d)


def shift_doublet(ev, d, dxy=(0.0, 0.0), dz=0.0):
    """Changes moving both hits of doublet d = (module, lo, up) rigidly."""
    P = points(ev)
    return {h: (P[h, 0] + dxy[0], P[h, 1] + dxy[1], P[h, 2] + dz) for h in (d[1], d[2])}


def rotate_upper(ev, d, direction_angle):
    """Change putting the upper hit of doublet d at the lower hit plus the same transverse
    length along azimuth ``direction_angle`` (z unchanged)."""
    P = points(ev)
    lo, up = P[d[1]], P[d[2]]
    L = np.hypot(up[0] - lo[0], up[1] - lo[1])
    return {d[2]: (lo[0] + L * np.cos(direction_angle), lo[1] + L * np.sin(direction_angle), up[2])}


def curvature(p, q, s):
    """Signed curvature of the circle through three transverse points (float64)."""
    ax, ay = p[0] - q[0], p[1] - q[1]
    cx, cy = s[0] - q[0], s[1] - q[1]
    cross = ax * cy - ay * cx
    return 2.0 * cross / (np.hypot(ax, ay) * np.hypot(cx, cy) * np.hypot(s[0] - p[0], s[1] - p[1]))


def md_row(r, d):
    """Index of doublet d's MD in the oracle's MD list (or None)."""
    md = r["md"]
    k = np.nonzero((md[:, 1] == d[1]) & (md[:, 2] == d[2]))[0]
    return int(k[0]) if len(k) else None


def has(r, key, mds):
    """Is the object made of these MD indices in list ``key`` of result r?"""
    if any(m is None for m in mds):
        return False
    rows = r[key]
    return bool(len(rows)) and bool(np.any(np.all(rows == np.array(mds, np.uint32), axis=1)))


def track_through(a1, a2, R, q, eta, like_centre):
    """Generator track of radius R and charge q whose circle passes through transverse
    points a1 and a2 (centre on the side of ``like_centre``), starting at its point of
    closest approach to the beam line, with z matching a1 at pseudorapidity eta."""
    a1, a2 = np.asarray(a1, np.float64), np.asarray(a2, np.float64)
    m = 0.5 * (a1[:2] + a2[:2])
    c = a2[:2] - a1[:2]
    n = np.array([-c[1], c[0]]) / np.hypot(*c)
    h = np.sqrt(R * R - 0.25 * np.dot(c, c))
    C = m + h * n if np.dot(m + h * n - like_centre, m + h * n - like_centre) < np.dot(m - h * n - like_centre, m - h * n - like_centre) else m - h * n
    v = C * (1.0 - R / np.hypot(*C))
    sin0, cos0 = (C[0] - v[0]) / (q * R), -(C[1] - v[1]) / (q * R)
    phi0 = np.arctan2(sin0, cos0)
    alpha1 = 2.0 * np.arcsin(np.hypot(*(a1[:2] - v)) / (2.0 * R))
    vz = a1[2] - R * alpha1 * np.sinh(eta)
    return track(R * S.PT_PER_CM, phi0, eta, q, (v[0], v[1], vz))
