"""Seeded synthetic events: helix tracks through the doublet geometry, noise hits, pixel seeds.

This is an *input generator*.  It simulates what the detector records -- the points where
charged helices cross sensor surfaces, smeared by the sensor resolution -- and it knows
nothing about how the tracking method pairs, links or selects those hits.  The CPU oracle
and the CUDA library both read its output.

Physics model (units cm, GeV, T):
  * Helix in B = 3.8 T along z: transverse radius R = pT / (0.0029979 * B).  A track of
    charge q, azimuth phi0 and pseudorapidity eta leaving vertex v follows
    p(alpha) = c + q R (-sin(phi0 - q alpha), cos(phi0 - q alpha)), z = v_z + R alpha sinh(eta),
    with centre c = v + q R (sin phi0, -cos phi0).  Only the first outgoing half turn
    (0 < alpha <= pi) records hits.
  * A hit is the exact crossing of a sensor surface (barrel cylinder or endcap plane),
    assigned to the module containing the crossing.  Resolution: 30 um along r-phi
    (a rotation about the beam line), barrel PS z smeared 0.5 mm, barrel 2S z replaced by
    the centre of its 2.5 cm strip, endcap r smeared 0.5 mm.  ``exact=True`` turns all
    of that off (points on the helix up to float32 rounding).  In the realistic geometry a
    tilted PS module measures its coarse coordinate along its own surface (0.5 mm, which
    moves both r and z), and a 2S endcap module gives r as the centre of a 5 cm strip.
  * Noise hits: a fraction of the track-hit count, each on a uniformly chosen module and
    sensor, uniform on the sensor area, with the same resolution model.
  * Pixel seeds (pLS): for every track with pT >= 0.8 GeV, four hits on pixel cylinders at
    r = 3, 7, 11, 16 cm (smeared 10 um in r-phi and z), and helix parameters at the first
    pixel hit with pT smeared by 1 % and phi by 1 mrad; plus 10 % fake seeds with random
    parameters and random hits.
Hit order is shuffled so that input order carries no information.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import geometry as G

SIGMA_RPHI = 0.003
SIGMA_Z_PS = 0.05
STRIP_2S = 2.5
SIGMA_R_EC = 0.05
PIXEL_R = (3.0, 7.0, 11.0, 16.0)
SIGMA_PIX = 0.001
PLS_PT_MIN = 0.8

PLS_DTYPE = np.dtype(
    [
        ("px", np.float32), ("py", np.float32), ("pz", np.float32),
        ("x0", np.float32), ("y0", np.float32), ("z0", np.float32),
        ("hx", np.float32, (4,)), ("hy", np.float32, (4,)), ("hz", np.float32, (4,)),
        ("charge", np.int32), ("n_hits", np.uint32),
    ]
)
assert PLS_DTYPE.itemsize == 80

TRACK_DTYPE = np.dtype(
    [("pt", np.float64), ("phi0", np.float64), ("eta", np.float64), ("q", np.int32),
     ("vx", np.float64), ("vy", np.float64), ("vz", np.float64)]
)


@dataclass
class Event:
    x: np.ndarray          # float32 [n_hits]
    y: np.ndarray
    z: np.ndarray
    det: np.ndarray        # uint32 [n_hits] = 2 * module + sensor (0 lower, 1 upper)
    sim: np.ndarray        # int32 [n_hits] generating track, -1 for noise
    tracks: np.ndarray     # TRACK_DTYPE [n_tracks]
    pls: np.ndarray = field(default_factory=lambda: np.zeros(0, PLS_DTYPE))
    pls_sim: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))

    @property
    def n_hits(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_pls(self) -> int:
        return int(self.pls.shape[0])


def helix_centre(t):
    R = t["pt"] / G.PT_PER_CM
    q = t["q"].astype(np.float64)
    cx = t["vx"] + q * R * np.sin(t["phi0"])
    cy = t["vy"] - q * R * np.cos(t["phi0"])
    return R, q, cx, cy


def helix_point(t, alpha):
    R, q, cx, cy = helix_centre(t)
    ph = t["phi0"] - q * alpha
    x = cx - q * R * np.sin(ph)
    y = cy + q * R * np.cos(ph)
    z = t["vz"] + R * alpha * np.sinh(t["eta"])
    return x, y, z, ph


def cylinder_alpha(t, rho):
    """Smallest turning angle in (0, pi] at which each track crosses r = rho outward (nan: none)."""
    R, q, cx, cy = helix_centre(t)
    D = np.hypot(cx, cy)
    K = (rho * rho - D * D - R * R) / (2.0 * q * R)
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = K / D
        psi = np.arctan2(-cx, cy)
        ac = np.arccos(np.clip(ratio, -1.0, 1.0))
    best = np.full(R.shape, np.nan)
    for sgn in (1.0, -1.0):
        ph = psi + sgn * ac
        alpha = np.mod(q * (t["phi0"] - ph), 2 * np.pi)
        x = cx - q * R * np.sin(ph)
        y = cy + q * R * np.cos(ph)
        outgoing = x * np.cos(ph) + y * np.sin(ph) > 0
        ok = (np.abs(ratio) <= 1.0) & (alpha > 0) & (alpha <= np.pi) & outgoing
        better = ok & (np.isnan(best) | (alpha < best))
        best = np.where(better, alpha, best)
    return best


def plane_alpha(t, zp):
    R = t["pt"] / G.PT_PER_CM
    sh = np.sinh(t["eta"])
    with np.errstate(invalid="ignore", divide="ignore"):
        alpha = (zp - t["vz"]) / (R * sh)
    ok = np.isfinite(alpha) & (alpha > 0) & (alpha <= np.pi)
    return np.where(ok, alpha, np.nan)


STRIP_2S_EC = 5.0  # radial strip length of a 2S endcap module (realistic geometry)


def cone_alpha(t, r0, zc, tilt, offset):
    """Turning angle in (0, pi] at which each track crosses, moving outward, the surface
    (r - r0) cos(tilt) + (z - zc) sin(tilt) = offset (a tilted module's sensor plane in
    r-z, a cone about the beam line); nan where it does not.  Bisection on the helix."""
    ct, st = np.cos(tilt), np.sin(tilt)

    def f(a):
        x, y, z, _ = helix_point(t, a)
        return (np.hypot(x, y) - r0) * ct + (z - zc) * st - offset

    R = t["pt"] / G.PT_PER_CM
    lo = np.full(len(t), 1e-9)
    hi = cylinder_alpha(t, r0 + 12.0)
    hi = np.where(np.isnan(hi), np.pi, hi)
    flo, fhi = f(lo), f(hi)
    ok = (flo < 0) & (fhi > 0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        up = fm > 0
        hi = np.where(up, mid, hi)
        lo = np.where(up, lo, mid)
    a = 0.5 * (lo + hi)
    x0, y0, _, _ = helix_point(t, a)
    x1, y1, _, _ = helix_point(t, np.minimum(a + 1e-6, np.pi))
    outward = np.hypot(x1, y1) >= np.hypot(x0, y0)
    return np.where(ok & outward & (R > 0), a, np.nan)


def _smear(rng, geom: G.Geometry, x, y, z, module, exact):
    """Apply the sensor resolution model to float64 points on their modules."""
    if exact or x.size == 0:
        return x, y, z
    m = geom.modules[module]
    barrel = m["subdet"] == G.SUBDET_BARREL
    r = np.hypot(x, y)
    d = rng.normal(0.0, SIGMA_RPHI, size=x.shape) / r
    c, s = np.cos(d), np.sin(d)
    x, y = x * c - y * s, x * s + y * c
    ps = m["stype"] == G.STYPE_PS
    tilt = m["tilt"].astype(np.float64)
    # PS: the coarse coordinate along the module surface in the r-z plane, (-sin t, cos t)
    ds = rng.normal(0.0, SIGMA_Z_PS, size=z.shape)
    zs = z + np.cos(tilt) * ds
    rs = r - np.sin(tilt) * ds
    zq = (np.floor(z / STRIP_2S) + 0.5) * STRIP_2S
    z = np.where(barrel, np.where(ps, zs, zq), z)
    r_ec_ps = r + rng.normal(0.0, SIGMA_R_EC, size=r.shape)
    emin = m["emin"].astype(np.float64)
    r_ec_2s = emin + (np.floor((r - emin) / STRIP_2S_EC) + 0.5) * STRIP_2S_EC
    rnew = np.where(barrel, np.where(ps, rs, r), np.where(ps, r_ec_ps, r_ec_2s))
    scale = rnew / r
    return x * scale, y * scale, z


def track_crossings(geom: G.Geometry, t):
    """All sensor crossings of tracks ``t``: (track, alpha, module, sensor, x, y, z) float64."""
    out = []
    n = len(t)
    idx = np.arange(n)
    zr_cache = {}
    for li in range(len(G.BARREL_R)):
        tilted_rows = [iz for iz in range(G.BARREL_NZ) if geom.row_tilt[(li + 1, iz)] != 0.0]
        for sensor in (0, 1):
            rho = G.BARREL_R[li] + sensor * G.BARREL_GAP[li]
            a = cylinder_alpha(t, rho)
            ok = ~np.isnan(a)
            if np.any(ok):
                tt = t[ok]
                x, y, z, _ = helix_point(tt, a[ok])
                mod = geom.barrel_module(np.full(len(tt), li + 1), z, np.arctan2(y, x))
                keep = mod >= 0
                if tilted_rows:  # cylinder crossings count only on flat rows
                    keep &= geom.modules["tilt"][np.maximum(mod, 0)] == 0.0
                out.append((idx[ok][keep], a[ok][keep], mod[keep], np.full(keep.sum(), sensor),
                            x[keep], y[keep], z[keep]))
            # tilted rows: the crossing of each row's section (upper sensor one gap along
            # the module normal), kept where it lies between the rays from the origin
            # through the row's z-bin edges at the layer radius; every (track, row) pair
            # that can meet is solved at once
            if tilted_rows:
                r0 = G.BARREL_R[li]
                gap = G.BARREL_GAP[li]
                pairs_t, pairs_row = [], []
                for iz in tilted_rows:
                    tilt = geom.row_tilt[(li + 1, iz)]
                    z_lo = -G.BARREL_ZHALF + iz * G.BARREL_ZLEN
                    span = G.BARREL_ZLEN * abs(np.tan(tilt))
                    zr = zr_cache.get((li, round(span, 6)))
                    if zr is None:
                        a1 = cylinder_alpha(t, max(r0 - span, 1.0))
                        a2 = cylinder_alpha(t, r0 + span + gap)
                        _, _, z1, _ = helix_point(t, np.where(np.isnan(a1), 0.0, a1))
                        _, _, z2, _ = helix_point(t, np.where(np.isnan(a2), np.pi, a2))
                        zr = (~np.isnan(a1), np.minimum(z1, z2), np.maximum(z1, z2))
                        zr_cache[(li, round(span, 6))] = zr
                    cand = np.nonzero(zr[0] & (zr[2] > z_lo - 5.0) & (zr[1] < z_lo + G.BARREL_ZLEN + 5.0))[0]
                    pairs_t.append(cand)
                    pairs_row.append(np.full(len(cand), iz))
                ti = np.concatenate(pairs_t)
                rows_i = np.concatenate(pairs_row)
                if len(ti):
                    tilt = np.array([geom.row_tilt[(li + 1, iz)] for iz in rows_i])
                    z_lo = -G.BARREL_ZHALF + rows_i * G.BARREL_ZLEN
                    zc = z_lo + 0.5 * G.BARREL_ZLEN
                    tt = t[ti]
                    a = cone_alpha(tt, r0, zc, tilt, sensor * gap)
                    ok = ~np.isnan(a)
                    x, y, z, _ = helix_point(tt[ok], a[ok])
                    tl, zlo, zcc = tilt[ok], z_lo[ok], zc[ok]
                    rl = np.hypot(x, y) - sensor * gap * np.cos(tl)  # the lower-sensor point
                    zl = z - sensor * gap * np.sin(tl)
                    inside = (zl * r0 >= zlo * rl) & (zl * r0 < (zlo + G.BARREL_ZLEN) * rl)
                    mod = geom.barrel_module(np.full(len(x), li + 1), zcc, np.arctan2(y, x))
                    keep = inside & (mod >= 0)
                    out.append((idx[ti][ok][keep], a[ok][keep], mod[keep], np.full(keep.sum(), sensor),
                                x[keep], y[keep], z[keep]))
    if not geom.barrel_only:
        for side in (-1, 1):
            for di, zd in enumerate(G.DISK_Z):
                for sensor in (0, 1):
                    zp = side * (zd + sensor * G.DISK_GAP)
                    a = plane_alpha(t, zp)
                    ok = ~np.isnan(a)
                    if not np.any(ok):
                        continue
                    tt = t[ok]
                    x, y, z, _ = helix_point(tt, a[ok])
                    mod = geom.endcap_module(side, di + 1, np.hypot(x, y), np.arctan2(y, x))
                    keep = mod >= 0
                    out.append((idx[ok][keep], a[ok][keep], mod[keep], np.full(keep.sum(), sensor),
                                x[keep], y[keep], np.full(keep.sum(), zp)))
    if not out:
        e = np.zeros(0)
        return (e.astype(np.int64), e, e.astype(np.int64), e.astype(np.int64), e, e, e)
    cols = [np.concatenate([o[i] for o in out]) for i in range(7)]
    order = np.lexsort((cols[1], cols[0]))
    return tuple(c[order] for c in cols)


def noise_points(rng, geom: G.Geometry, n):
    """``n`` hits uniform over modules, sensors and module area (float64 points)."""
    if n <= 0:
        e = np.zeros(0)
        return e, e, e, e.astype(np.int64), e.astype(np.int64)
    mod = rng.integers(0, geom.n_modules, size=n)
    sensor = rng.integers(0, 2, size=n)
    m = geom.modules[mod]
    barrel = m["subdet"] == G.SUBDET_BARREL
    k = m["iphi"].astype(np.float64)
    nphi = m["nphi"].astype(np.float64)
    phi = 2 * np.pi * (k + rng.random(n)) / nphi
    u = rng.random(n)
    ext = m["emin"] + u * (m["emax"] - m["emin"])
    surf = m["surf"].astype(np.float64) + sensor * m["gap"] * np.where(barrel, 1.0, m["side"])
    r = np.where(barrel, surf, ext)
    z = np.where(barrel, ext, surf)
    # tilted barrel modules: uniform along the row's section between the rays from the
    # origin through the bin edges, the upper sensor one gap along the normal
    tilt = m["tilt"].astype(np.float64)
    r0 = m["surf"].astype(np.float64)
    zlo, zhi = m["emin"].astype(np.float64), m["emax"].astype(np.float64)
    zc = 0.5 * (zlo + zhi)
    ct, st = np.cos(tilt), np.sin(tilt)
    u_lo = (zlo - zc) / (ct + zlo / r0 * st)
    u_hi = (zhi - zc) / (ct + zhi / r0 * st)
    w = u_lo + rng.random(n) * (u_hi - u_lo)
    r = np.where(tilt != 0.0, r0 - w * st + sensor * m["gap"] * ct, r)
    z = np.where(tilt != 0.0, zc + w * ct + sensor * m["gap"] * st, z)
    return r * np.cos(phi), r * np.sin(phi), z, mod, sensor


def make_pls(rng, t, track_ids, n_fake, exact=False, triplet_frac=0.0):
    """Pixel seeds for tracks ``t`` (already selected) plus ``n_fake`` random seeds.

    ``exact`` keeps the hits on the helix and the parameters unsmeared.  A fraction
    ``triplet_frac`` of the seeds lose one of their four pixel hits (chosen at random):
    triplets, whose three hits come first, whose fourth slot is zero, and whose reference
    point and direction are those at their first remaining hit."""
    w = 0.0 if exact else 1.0
    n = len(t)
    alphas = np.stack([cylinder_alpha(t, r) for r in PIXEL_R], axis=1) if n else np.zeros((0, 4))
    ok = ~np.any(np.isnan(alphas), axis=1) if n else np.zeros(0, bool)
    t = t[ok]
    alphas = alphas[ok]
    track_ids = track_ids[ok]
    n = len(t)
    pls = np.zeros(n + n_fake, PLS_DTYPE)
    sim = np.concatenate([track_ids.astype(np.int32), np.full(n_fake, -1, np.int32)])
    if n:
        hx = np.zeros((n, 4)); hy = np.zeros((n, 4)); hz = np.zeros((n, 4))
        for k in range(4):
            x, y, z, _ = helix_point(t, alphas[:, k])
            d = w * rng.normal(0.0, SIGMA_PIX, size=n) / PIXEL_R[k]
            c, s = np.cos(d), np.sin(d)
            hx[:, k] = x * c - y * s
            hy[:, k] = x * s + y * c
            hz[:, k] = z + w * rng.normal(0.0, SIGMA_PIX, size=n)
        q = t["q"].astype(np.float64)
        dphi = w * rng.normal(0.0, 0.001, size=n)
        phi1 = t["phi0"] - q * alphas[:, 0] + dphi
        pt = t["pt"] * (1.0 + w * rng.normal(0.0, 0.01, size=n))
        pls["px"][:n] = pt * np.cos(phi1)
        pls["py"][:n] = pt * np.sin(phi1)
        pls["pz"][:n] = pt * np.sinh(t["eta"])
        pls["hx"][:n] = hx; pls["hy"][:n] = hy; pls["hz"][:n] = hz
        pls["x0"][:n] = pls["hx"][:n, 0]; pls["y0"][:n] = pls["hy"][:n, 0]; pls["z0"][:n] = pls["hz"][:n, 0]
        pls["charge"][:n] = t["q"]
    if n_fake:
        f = slice(n, n + n_fake)
        pt = np.minimum(PLS_PT_MIN / (1.0 - rng.random(n_fake)), 200.0)
        phi = rng.uniform(0, 2 * np.pi, n_fake)
        eta = rng.uniform(-2.4, 2.4, n_fake)
        pls["px"][f] = pt * np.cos(phi)
        pls["py"][f] = pt * np.sin(phi)
        pls["pz"][f] = pt * np.sinh(eta)
        hphi = rng.uniform(0, 2 * np.pi, (n_fake, 4))
        for k in range(4):
            pls["hx"][f, k] = PIXEL_R[k] * np.cos(hphi[:, k])
            pls["hy"][f, k] = PIXEL_R[k] * np.sin(hphi[:, k])
            pls["hz"][f, k] = rng.uniform(-30, 30, n_fake)
        pls["x0"][f] = pls["hx"][f, 0]; pls["y0"][f] = pls["hy"][f, 0]; pls["z0"][f] = pls["hz"][f, 0]
        pls["charge"][f] = rng.choice(np.array([-1, 1], np.int32), n_fake)
    pls["n_hits"] = 4
    if triplet_frac > 0.0 and len(pls):
        drop = rng.integers(0, 4, len(pls))
        trip = np.nonzero(rng.random(len(pls)) < triplet_frac)[0]
        for i in trip:
            keep = [k for k in range(4) if k != drop[i]]
            for key in ("hx", "hy", "hz"):
                pls[key][i] = np.concatenate([pls[key][i][keep], [0.0]])
            pls["n_hits"][i] = 3
            pls["x0"][i], pls["y0"][i], pls["z0"][i] = pls["hx"][i][0], pls["hy"][i][0], pls["hz"][i][0]
            if i < n and drop[i] == 0:  # the reference moves to the second pixel layer
                ptr = float(np.hypot(pls["px"][i], pls["py"][i]))
                ph = t["phi0"][i] - q[i] * alphas[i, 1] + dphi[i]
                pls["px"][i], pls["py"][i] = ptr * np.cos(ph), ptr * np.sin(ph)
    return pls, sim


def event_from_tracks(geom: G.Geometry, t, seed: int, *, noise_frac=0.0, exact=False,
                      with_pls=False, fake_pls_frac=0.10, shuffle=True, triplet_frac=0.0) -> Event:
    """Simulate the hits (and optionally the pixel seeds) of the given tracks."""
    rng = np.random.default_rng(seed)
    trk, _alpha, mod, sensor, x, y, z = track_crossings(geom, t)
    x, y, z = _smear(rng, geom, x, y, z, mod, exact)
    n_noise = int(round(noise_frac * len(x)))
    nx, ny, nz, nmod, nsen = noise_points(rng, geom, n_noise)
    nx, ny, nz = _smear(rng, geom, nx, ny, nz, nmod, exact)
    X = np.concatenate([x, nx]); Y = np.concatenate([y, ny]); Z = np.concatenate([z, nz])
    det = np.concatenate([2 * mod + sensor, 2 * nmod + nsen]).astype(np.uint32)
    sim = np.concatenate([trk, np.full(n_noise, -1)]).astype(np.int32)
    if shuffle:
        perm = rng.permutation(len(X))
        X, Y, Z, det, sim = X[perm], Y[perm], Z[perm], det[perm], sim[perm]
    ev = Event(X.astype(np.float32), Y.astype(np.float32), Z.astype(np.float32), det, sim, t)
    if with_pls:
        sel = np.nonzero(t["pt"] >= PLS_PT_MIN)[0]
        n_fake = int(round(fake_pls_frac * len(sel)))
        ev.pls, ev.pls_sim = make_pls(rng, t[sel], sel, n_fake, exact=exact, triplet_frac=triplet_frac)
    return ev


def random_tracks(rng, n, *, pt_mode="uniform", pt_lo=1.0, pt_hi=10.0, eta_max=1.0,
                  sigma_z0=5.0, pt_cap=200.0):
    """Prompt tracks from the beam spot: ``uniform`` pT in [lo, hi] or ``inv2`` (pdf ~ 1/pT^2 above lo)."""
    t = np.zeros(n, TRACK_DTYPE)
    if pt_mode == "uniform":
        t["pt"] = rng.uniform(pt_lo, pt_hi, n)
    else:
        t["pt"] = np.minimum(pt_lo / (1.0 - rng.random(n)), pt_cap)
    t["phi0"] = rng.uniform(-np.pi, np.pi, n)
    t["eta"] = rng.uniform(-eta_max, eta_max, n)
    t["q"] = rng.choice(np.array([-1, 1], np.int32), n)
    t["vz"] = rng.normal(0.0, sigma_z0, n)
    return t
