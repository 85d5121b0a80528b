"""Pins of the oracle on the geometry with tilted inner-barrel modules (Fig. 1).

In layers 1-3 the rows with |z| >= 45 cm are tilted towards the interaction point; a
tilted PS module's sensors are sections of cones about the beam line, the upper sensor one
gap along the module normal, and its coarse coordinate runs along its surface, so its
hits carry both a z and a radial tolerance.  The cut forms are the same; these pins check
that the module constants, the connection map and the chain handle such modules: noiseless
tracks through tilted modules keep every MD, LS and T5 they should, a hit moved along the
tilted surface is accepted or rejected at the resolution the reading gives, the map loses
no LS, and the joins equal brute force.
"""
import numpy as np

import lst_synth as S
import oracle
from lst_synth import events as E
from helix_cases import doublets, edited, event, md_row, points, track


def test_tilted_hits_lie_on_their_sections(tilted_geom):
    """Generator pin: every hit of a tilted module lies on its cone section (upper sensor
    one gap along the normal) between the rays through its z-bin edges."""
    ev = S.make_event("pu200", 0, n_tracks=1500, realistic=True, exact=True)
    m = tilted_geom.modules[ev.det >> 1]
    sel = m["tilt"] != 0
    assert sel.sum() > 500
    up = (ev.det & 1)[sel].astype(np.float64)
    t = m["tilt"][sel].astype(np.float64)
    r = np.hypot(ev.x[sel], ev.y[sel]).astype(np.float64)
    z = ev.z[sel].astype(np.float64)
    zc = 0.5 * (m["emin"][sel] + m["emax"][sel])
    res = (r - m["surf"][sel]) * np.cos(t) + (z - zc) * np.sin(t) - up * m["gap"][sel]
    assert np.max(np.abs(res)) < 2e-5
    rl, zl = r - up * m["gap"][sel] * np.cos(t), z - up * m["gap"][sel] * np.sin(t)
    track_hits = ev.sim[sel] >= 0
    lo_ray = zl * m["surf"][sel] - m["emin"][sel] * rl
    hi_ray = zl * m["surf"][sel] - m["emax"][sel] * rl
    assert np.all(lo_ray[track_hits] >= -1e-3) and np.all(hi_ray[track_hits] <= 1e-3)


def _adjacent(mods, a, b):
    """b's surface is next to a's (barrel layer -> next layer or first disk; disk -> next disk)."""
    ma, mb = mods[a], mods[b]
    if ma["subdet"] == 0:
        return (mb["subdet"] == 0 and mb["layer"] == ma["layer"] + 1) or (mb["subdet"] == 1 and mb["layer"] == 1)
    return mb["subdet"] == 1 and mb["side"] == ma["side"] and mb["layer"] == ma["layer"] + 1


def test_noiseless_tracks_through_tilted_modules(tilted_geom, ora_tilted):
    """Every noiseless 1-10 GeV track crossing tilted modules gives an MD on each module
    where both its sensor hits landed, the LS between each pair of such MDs on surfaces it
    crosses one after the other, and a T5 when five such MDs follow one another."""
    rng = np.random.default_rng(71)
    t = E.random_tracks(rng, 160, pt_mode="uniform", pt_lo=1.0, pt_hi=10.0, eta_max=1.6)
    t["eta"] = np.sign(t["eta"]) * (0.85 + np.abs(t["eta"]) * (0.75 / 1.6))
    mods = tilted_geom.modules
    n_tilted = n_t5 = 0
    for i in range(len(t)):
        ev = event(tilted_geom, t[i:i + 1])
        d = doublets(ev)
        if not any(mods["tilt"][x[0]] != 0 for x in d):
            continue
        r = oracle.run(ora_tilted, ev)
        mds = [md_row(r, x) for x in d]
        assert None not in mds, i
        n_tilted += 1
        ls = {tuple(map(int, x)) for x in r["ls"]}
        # hits come in crossing order: an LS is due between two clean doublets when no
        # other sensor crossing lies between them
        consecutive = [d[k + 1][1] == d[k][2] + 1 and _adjacent(mods, d[k][0], d[k + 1][0])
                       for k in range(len(d) - 1)]
        for k in range(len(d) - 1):
            if consecutive[k]:
                assert (mds[k], mds[k + 1]) in ls, (i, k)
        if any(all(consecutive[k0:k0 + 4]) for k0 in range(len(d) - 4)):
            n_t5 += 1
            assert len(r["t5"]) >= 1, i
    assert n_tilted > 60 and n_t5 > 30


def _tilted_track(tilted_geom, layer):
    for phi0 in np.linspace(0.11, 6.1, 41):
        for eta in (1.45, 1.2, 0.95):
            ev = event(tilted_geom, track(3.0, phi0, eta))
            for x in doublets(ev):
                m = tilted_geom.modules[x[0]]
                if m["subdet"] == 0 and m["layer"] == layer and m["tilt"] != 0:
                    return ev, x
    raise AssertionError


def test_tilted_md_window_along_the_surface(tilted_geom, ora_tilted):
    """A tilted PS module measures its coarse coordinate along its surface to 0.5 mm
    (3 sigma = 0.15 cm per hit): the pair's r-z pointing tolerates moving the upper hit
    along the surface by about 2 x 0.15 cm plus the luminous region seen over the gap.
    1.5 x that: no MD; 0.5 x: the MD is there."""
    for layer in (1, 2, 3):
        ev, d = _tilted_track(tilted_geom, layer)
        m = tilted_geom.modules[d[0]]
        t = float(m["tilt"])
        P = points(ev)
        lo, up = P[d[1]], P[d[2]]
        ra, rb = np.hypot(*lo[:2]), np.hypot(*up[:2])
        zb = up[2]
        # |d f / d s| of f = z_a r_b - r_a z_b for a move ds along (-sin t, cos t) in (r, z)
        slope = abs(lo[2] * np.sin(t) + ra * np.cos(t))
        tol = (15.0 * abs(rb - ra) + 0.15 * abs(np.cos(t)) * (ra + rb) + 0.15 * abs(np.sin(t)) * (abs(lo[2]) + abs(zb)))
        allowed = tol / slope
        for f, present in ((1.5, False), (0.5, True)):
            s = -np.sign(lo[2] * rb - ra * zb) if (lo[2] * rb - ra * zb) != 0 else 1.0
            ds = s * f * allowed
            rn = rb - np.sin(t) * ds
            new = (up[0] * rn / rb, up[1] * rn / rb, zb + np.cos(t) * ds)
            e2 = edited(ev, {d[2]: new})
            assert oracle.md_test(ora_tilted, d[0], points(e2)[d[1]], points(e2)[d[2]]) == present, (layer, f)
            r = oracle.run(ora_tilted, e2)
            assert (md_row(r, d) is not None) == present, (layer, f)


def test_tilted_doublets_with_resolution(tilted_geom, ora_tilted):
    """With the along-surface resolution, >= 95 % of the reachable true MDs on tilted
    modules survive, and >= 90 % of the tracks with both sensor hits on five or more
    modules are matched by a candidate (75 % rule, Sec. 3)."""
    rng = np.random.default_rng(72)
    t = E.random_tracks(rng, 500, pt_mode="uniform", pt_lo=1.0, pt_hi=10.0, eta_max=1.6)
    t["eta"] = np.sign(t["eta"]) * (0.85 + np.abs(t["eta"]) * (0.75 / 1.6))
    ev = E.event_from_tracks(tilted_geom, t, 72, exact=False)
    r = oracle.run(ora_tilted, ev)
    mods = tilted_geom.modules
    md = r["md"]
    tilted = mods["tilt"][md[:, 0]] != 0
    true_md = ev.sim[md[:, 1]] == ev.sim[md[:, 2]]
    on_t = mods["tilt"][ev.det >> 1] != 0
    key = ev.sim.astype(np.int64) * 100000 + (ev.det >> 1)
    u, c = np.unique(key[on_t], return_counts=True)
    reachable = int((c == 2).sum())
    assert reachable > 400
    assert (true_md & tilted).sum() >= 0.95 * reachable
    matched = set()
    for ot in r["tc_ot"]:
        h = ot[ot != 0xFFFFFFFF]
        s_, n_ = np.unique(ev.sim[h], return_counts=True)
        if n_.max() > 0.75 * len(h) and s_[n_.argmax()] >= 0:
            matched.add(int(s_[n_.argmax()]))
    # tracks that can form a T5: both sensor hits on at least five modules
    k_all, c_all = np.unique(key[ev.sim >= 0], return_counts=True)
    per_track = np.bincount((k_all[c_all == 2] // 100000).astype(np.int64), minlength=len(t))
    reach = set(np.nonzero(per_track >= 5)[0].tolist())
    assert len(reach) > 300
    assert len(matched & reach) >= 0.9 * len(reach)


def test_tilted_connection_map_loses_no_ls(ora_tilted):
    """The map's box for a tilted module spans its section: no LS is lost against
    testing every MD pair on adjacent surfaces."""
    for n, i in ((600, 1), (1500, 2)):
        ev = S.make_event("pu200", i, n_tracks=n, realistic=True)
        a = oracle.run(ora_tilted, ev)
        b = oracle.run(ora_tilted, ev, brute_ls=True)
        assert len(a["ls"]) > 0
        assert np.array_equal(a["ls"], b["ls"]) and np.array_equal(a["t5"], b["t5"])


def test_tilted_modules_keep_the_pt_threshold(tilted_geom, ora_tilted):
    """The bending slope of a tilted module comes from its largest radius (its section
    spans surf +- half its z length x |tan(tilt)|): prompt tracks 0.5 % above 0.8 GeV (Sec. 1)
    through tilted modules keep every MD and every LS between MDs they cross one after the
    other."""
    n = 0
    # tracks that cross a tilted section low in its z bin, where the section lies above
    # the layer radius (and needs the span in the slope), plus a few elsewhere
    etas = [float(np.arcsinh(z / r)) for r in (23.0, 36.0, 51.0) for z in (40.2, 50.2, 60.2)]
    for eta in etas + [-e for e in etas[::3]] + [1.25, 1.5]:
        for phi0 in np.linspace(0.2, 6.0, 9):
            for q in (-1, 1):
                ev = event(tilted_geom, track(0.8 * 1.005, phi0, eta, q))
                d = doublets(ev)
                if not any(tilted_geom.modules["tilt"][x[0]] != 0 for x in d):
                    continue
                r = oracle.run(ora_tilted, ev)
                mds = [md_row(r, x) for x in d]
                assert None not in mds
                ls = {tuple(map(int, x)) for x in r["ls"]}
                for k in range(len(d) - 1):
                    if d[k + 1][1] == d[k][2] + 1 and _adjacent(tilted_geom.modules, d[k][0], d[k + 1][0]):
                        assert (mds[k], mds[k + 1]) in ls
                        n += 1
    assert n > 60
