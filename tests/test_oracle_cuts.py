"""Rejection side of every oracle cut, on noiseless helices with one doublet or one seed
parameter moved.

Each case is built so that one named condition of the reading decides: moved beyond its
bound (by a factor taken from the geometry, in float64 here) the object must be missing
from the whole chain's output and the predicate-level evaluation must show that condition,
and only it, failing; moved by a fraction of the bound (the mirrored case) the object must
be there.  The amounts come from the geometry of the readings (paper Sec. 1: pT >= 0.8
GeV windows, objects built from MDs on connected modules, T5s without a beam-line cut),
not from the oracle's expressions, and the margins leave the float32 rounding out of it.
"""
import numpy as np
import pytest

import oracle
from oracle import (LS_BEND, LS_DIR_IN, LS_DIR_OUT, LS_EXIT, LS_RZ, PLS_RPHI, PLS_RZ, PT5_CURV, PT5_WINDOWS,
                    T3_MIDDIR, T3_RADIUS, T3_RZ, T5_BRFULL, T5_INOUT, T5_RADIUS, T5_RZ)
from helix_cases import (EDIR, RMIN, clean_track, curvature, doublets, edited, event, has, md_row, outward,
                         points, rotate_upper, shift_doublet, track, track_through)

ALL_LS = LS_BEND | LS_RZ | LS_EXIT | LS_DIR_IN | LS_DIR_OUT
ALL_T3 = T3_RZ | T3_MIDDIR | T3_RADIUS
ALL_T5 = T5_INOUT | T5_BRFULL | T5_RADIUS | T5_RZ


def _ls_mask(og, ev, da, db):
    P = points(ev)
    return oracle.ls_eval(og, da[0], db[0], P[da[1]], P[da[2]], P[db[1]], P[db[2]])


def _t3_mask(og, ev, da, db, dc):
    P = points(ev)
    return oracle.t3_eval(og, (da[0], db[0], dc[0]), P[da[1]], P[db[1]], P[db[2]], P[dc[1]])


def _t5(og, ev, ds):
    P = points(ev)
    return oracle.t5_eval(og, [d[0] for d in ds], [P[d[1]] for d in ds])


def _mds(r, ds):
    return [md_row(r, d) for d in ds]


# ---------------------------------------------------------------- MD: r-z of the hit pair
def test_md_rz_rejects_upper_hit_moved_in_z(barrel_geom, ora_barrel):
    """Layer 1 (PS, 0.5 mm z resolution, 1.6 mm gap): a prompt pair can step in z by the
    luminous region seen over the gap (15 cm x 0.16 / 23) plus three sigma of both hits,
    about 0.4 cm.  1.5 x that: no MD; 0.4 x: the MD is there."""
    t, ev, d = clean_track(barrel_geom, 3.0, 0.2, 6)
    P = points(ev)
    lo, up = d[0][1], d[0][2]
    allowed = 15.0 * 0.16 / 23.0 + 3 * 0.05 * (1 + 23.16 / 23.0)
    for dz, present in ((1.5 * allowed, False), (0.4 * allowed, True)):
        e2 = edited(ev, {up: (P[up, 0], P[up, 1], P[up, 2] + dz)})
        assert oracle.md_test(ora_barrel, d[0][0], points(e2)[lo], points(e2)[up]) == present
        r = oracle.run(ora_barrel, e2)
        assert (md_row(r, d[0]) is not None) == present
        assert md_row(r, d[1]) is not None


# ---------------------------------------------------------------- LS
def test_ls_rz_rejects_vertex_outside_luminous_region(barrel_geom, ora_barrel):
    """The LS r-z line must point back to |z0| <= 15 cm (3 sigma of the luminous region)
    within the hits' z resolution (PS layers 1-2: about +0.7 cm).  z0 = 18 cm: no LS 1->2,
    only the r-z condition fails; z0 = 13 cm: the LS is there."""
    for z0, present in ((18.0, False), (13.0, True)):
        t, ev, d = clean_track(barrel_geom, 4.0, 0.3, 6, vz=z0)
        r = oracle.run(ora_barrel, ev)
        m = _mds(r, d)
        assert m[0] is not None and m[1] is not None       # both MDs exist either way
        assert has(r, "ls", (m[0], m[1])) == present
        mask = _ls_mask(ora_barrel, ev, d[0], d[1])
        assert mask == (ALL_LS if present else ALL_LS & ~LS_RZ)


def test_ls_bending_is_the_pt_threshold(barrel_geom, ora_barrel):
    """The LS bending window is the 0.8 GeV one (Sec. 1): a prompt track at 0.816 GeV
    keeps its layer 1->2 LS; at 0.72 GeV both MDs still form (the hit-pair window has the
    sensors' resolution) but the LS fails the bending condition alone."""
    for pt, present in ((0.8 * 1.02, True), (0.8 * 0.9, False)):
        t, ev, d = clean_track(barrel_geom, pt, 0.1, 6 if present else 5)
        r = oracle.run(ora_barrel, ev)
        m = _mds(r, d)
        assert m[0] is not None and m[1] is not None
        assert has(r, "ls", (m[0], m[1])) == present
        assert _ls_mask(ora_barrel, ev, d[0], d[1]) == (ALL_LS if present else ALL_LS & ~LS_BEND)


@pytest.mark.parametrize("which", ["outer", "inner"])
def test_ls_md_direction_rejects_rotated_md(barrel_geom, ora_barrel, which):
    """An MD's direction (upper - lower hit) is the local tangent; on a circle of radius
    R >= Rmin it differs from the LS chord c by at most asin(|c| / 2 Rmin), plus the
    direction error of an MD, EDIR / |d|.  Rotating the layer-3 MD (outer end of LS 2->3, or
    inner end of LS 3->4) to 1.3 x that bound from the chord removes the LS and only the
    direction condition of that MD fails; at 0.5 x the LS stays."""
    t, ev, d = clean_track(barrel_geom, 3.0, 0.25, 6)
    P = points(ev)
    da, db = (d[1], d[2]) if which == "outer" else (d[2], d[3])
    md = d[2]
    c = P[db[1], :2] - P[da[1], :2]
    clen = np.hypot(*c)
    dl = np.hypot(*(P[md[2], :2] - P[md[1], :2]))
    bound = np.arcsin(clen / (2 * RMIN)) + np.arcsin(EDIR / dl)
    chord_ang = np.arctan2(c[1], c[0])
    for f, present in ((1.3, False), (0.5, True)):
        ok = None
        for sgn in (1.0, -1.0):  # the side on which the MD itself still passes its window
            e2 = edited(ev, rotate_upper(ev, md, chord_ang + sgn * f * bound))
            if oracle.md_test(ora_barrel, md[0], points(e2)[md[1]], points(e2)[md[2]]):
                ok = e2
                break
        assert ok is not None
        r = oracle.run(ora_barrel, ok)
        m = _mds(r, (da, db))
        assert m[0] is not None and m[1] is not None
        assert has(r, "ls", m) == present
        bit = LS_DIR_OUT if which == "outer" else LS_DIR_IN
        assert _ls_mask(ora_barrel, ok, da, db) == (ALL_LS if present else ALL_LS & ~bit)


def test_ls_barrel_exit_rejects_skipped_layer(full_geom, ora_full):
    """A barrel-to-disk LS is only possible when the track leaves the barrel (|z| = 120)
    before the next barrel layer: with cot(theta) = 1.36 a prompt straight track crosses
    layer 5 (r = 86) at z = 117, so the layer 4 -> disk 1 LS must not exist (only the exit
    condition fails); with cot(theta) = 1.40 it misses layer 5 and the LS is there."""
    mods = full_geom.modules
    for cot, present in ((1.36, False), (1.40, True)):
        eta = np.arcsinh(cot)
        found = None
        for phi0 in np.linspace(0.13, 6.1, 37):
            t = track(10.0, phi0, eta, 1)
            ev = event(full_geom, t)
            d = doublets(ev)
            l4 = [x for x in d if mods[x[0]]["subdet"] == 0 and mods[x[0]]["layer"] == 4]
            d1 = [x for x in d if mods[x[0]]["subdet"] == 1 and mods[x[0]]["layer"] == 1]
            if l4 and d1:
                found = (ev, l4[0], d1[0], d)
                break
        assert found is not None
        ev, a, b, d = found
        hits5 = mods[ev.det >> 1]
        crosses5 = bool(np.any((hits5["subdet"] == 0) & (hits5["layer"] == 5)))
        assert crosses5 == (not present)
        r = oracle.run(ora_full, ev)
        m = _mds(r, (a, b))
        assert m[0] is not None and m[1] is not None
        assert has(r, "ls", m) == present
        assert _ls_mask(ora_full, ev, a, b) == (ALL_LS if present else ALL_LS & ~LS_EXIT)


# ---------------------------------------------------------------- T3
def test_t3_rz_rejects_middle_moved_in_z(barrel_geom, ora_barrel):
    """z is linear in arc length: the middle anchor of a triple may leave the a-c line by
    the z resolution of the three PS hits (0.15 cm each, about 0.3 cm in total).  1.0 cm
    removes T3 (1,2,3) with only the r-z condition failing (both LSs stay); 0.12 cm keeps
    it."""
    t, ev, d = clean_track(barrel_geom, 5.0, 0.2, 6)
    for dz, present in ((1.0, False), (0.12, True)):
        e2 = edited(ev, shift_doublet(ev, d[1], dz=dz))
        r = oracle.run(ora_barrel, e2)
        m = _mds(r, d[:3])
        assert has(r, "ls", (m[0], m[1])) and has(r, "ls", (m[1], m[2]))
        assert has(r, "t3", m) == present
        assert _t3_mask(ora_barrel, e2, *d[:3]) == (ALL_T3 if present else ALL_T3 & ~T3_RZ)


def test_t3_middle_direction_rejects_rotated_md(barrel_geom, ora_barrel):
    """On a circle the tangent at b and the chord a->c differ by half the difference of the
    arcs ab and bc (over 2 Rmin, with 2 % of |ac| slack) plus the MD's direction error.
    The layer-2 MD rotated to 1.35 x that bound from the chord removes T3 (1,2,3) while both
    LSs stay (their chord windows are wider); 0.5 x keeps it."""
    t, ev, d = clean_track(barrel_geom, 5.0, 0.2, 6)
    P = points(ev)
    a, b, c = P[d[0][1], :2], P[d[1][1], :2], P[d[2][1], :2]
    ac = c - a
    dab, dbc, dac = np.hypot(*(b - a)), np.hypot(*(c - b)), np.hypot(*ac)
    dl = np.hypot(*(P[d[1][2], :2] - P[d[1][1], :2]))
    bound = np.arcsin((abs(dbc - dab) + 0.02 * dac) / (2 * RMIN)) + np.arcsin(EDIR / dl)
    ang = np.arctan2(ac[1], ac[0])
    for f, present in ((1.35, False), (0.5, True)):
        done = False
        for sgn in (1.0, -1.0):
            e2 = edited(ev, rotate_upper(ev, d[1], ang + sgn * f * bound))
            r = oracle.run(ora_barrel, e2)
            m = _mds(r, d[:3])
            if not (has(r, "ls", (m[0], m[1])) and has(r, "ls", (m[1], m[2]))):
                continue
            assert has(r, "t3", m) == present
            assert _t3_mask(ora_barrel, e2, *d[:3]) == (ALL_T3 if present else ALL_T3 & ~T3_MIDDIR)
            done = True
            break
        assert done


def test_t3_radius_threshold(barrel_geom, ora_barrel):
    """T3 radius >= 0.95 Rmin (Rmin: 0.8 GeV): the anchors of a 0.72 GeV helix (R = 0.9
    Rmin) fail only the radius condition; those of a 0.80 GeV helix pass all three."""
    for pt, ok in ((0.72, False), (0.80, True)):
        ev = event(barrel_geom, track(pt, 0.4, 0.1))
        d = doublets(ev)
        assert len(d) >= 3
        assert _t3_mask(ora_barrel, ev, *d[:3]) == (ALL_T3 if ok else ALL_T3 & ~T3_RADIUS)


# ---------------------------------------------------------------- T5
def _t5_case(barrel_geom):
    return clean_track(barrel_geom, 5.0, 0.2, 6)


def test_t5_inner_outer_curvature(barrel_geom, ora_barrel):
    """Inner (a,b,c) and outer (c,d,e) curvatures must agree.  Moving anchor a outward and
    anchor e inward, with e's move solved in float64 so that the full (a,c,e) curvature
    stays the same, changes k_in and k_out in opposite directions while k_br and k_full stay:
    at 1.3x the tolerance (5 % of the curvature sum, the point errors and 1e-4 / cm) T5
    (1..5) is gone and only the inner/outer condition fails; at 0.75x it is there."""
    from scipy.optimize import brentq
    t, ev, d = _t5_case(barrel_geom)
    P = points(ev)
    A = [P[x[1], :2] for x in d[:5]]
    na, ne = outward(t, A[0]), outward(t, A[4])
    k0 = curvature(A[0], A[2], A[4])
    kin0, kout0 = curvature(A[0], A[1], A[2]), curvature(A[2], A[3], A[4])
    # 5 % of the curvature sum, the curvature change of a 0.01 cm point error on each
    # triple's span (8 delta / span^2) and 1e-4 / cm
    tol = 0.05 * (abs(kin0) + abs(kout0)) + 0.08 / np.sum((A[0] - A[2]) ** 2) + 0.08 / np.sum((A[2] - A[4]) ** 2) + 1e-4

    def solve(ea):
        a2 = A[0] + ea * na
        ee = brentq(lambda x: curvature(a2, A[2], A[4] + x * ne) - k0, -50 * abs(ea) - 1, 50 * abs(ea) + 1)
        return ea, ee, abs(curvature(a2, A[1], A[2]) - curvature(A[2], A[3], A[4] + ee * ne))

    for target, present in ((1.3, False), (0.75, True)):
        ea = brentq(lambda x: solve(x)[2] - target * tol, 1e-4, 1.0)
        _, ee, _ = solve(ea)
        ch = shift_doublet(ev, d[0], dxy=ea * na)
        ch.update(shift_doublet(ev, d[4], dxy=ee * ne))
        e2 = edited(ev, ch)
        r = oracle.run(ora_barrel, e2)
        m = _mds(r, d[:5])
        assert has(r, "t3", m[:3]) and has(r, "t3", m[2:5])
        assert has(r, "t5", m) == present
        mask, _, _ = _t5(ora_barrel, e2, d[:5])
        assert mask == (ALL_T5 if present else ALL_T5 & ~T5_INOUT)


def test_t5_bridge_full_curvature(barrel_geom, ora_barrel):
    """Bridge (b,c,d) and full (a,c,e) curvatures must agree.  Moving b and d outward by
    amounts solved so that k_in and k_out grow equally leaves the inner/outer condition
    satisfied and lowers k_br: at 1.3x the tolerance T5 (1..5) is gone with only the
    bridge/full condition failing, at 0.75x it is there."""
    from scipy.optimize import brentq
    t, ev, d = _t5_case(barrel_geom)
    P = points(ev)
    A = [P[x[1], :2] for x in d[:5]]
    nb, nd = outward(t, A[1]), outward(t, A[3])
    kin0, kout0 = curvature(A[0], A[1], A[2]), curvature(A[2], A[3], A[4])
    kbr0, kfu0 = curvature(A[1], A[2], A[3]), curvature(A[0], A[2], A[4])
    tol = 0.05 * (abs(kbr0) + abs(kfu0)) + 0.08 / np.sum((A[1] - A[3]) ** 2) + 0.08 / np.sum((A[0] - A[4]) ** 2) + 1e-4

    def solve(eb):
        b2 = A[1] + eb * nb
        dk = curvature(A[0], b2, A[2]) - kin0
        ed = brentq(lambda x: curvature(A[2], A[3] + x * nd, A[4]) - kout0 - dk, -50 * abs(eb) - 1, 50 * abs(eb) + 1)
        return ed, abs(curvature(b2, A[2], A[3] + ed * nd) - kfu0)

    for target, present in ((1.3, False), (0.75, True)):
        eb = brentq(lambda x: solve(x)[1] - target * tol, 1e-4, 1.0)
        ed, _ = solve(eb)
        ch = shift_doublet(ev, d[1], dxy=eb * nb)
        ch.update(shift_doublet(ev, d[3], dxy=ed * nd))
        e2 = edited(ev, ch)
        r = oracle.run(ora_barrel, e2)
        m = _mds(r, d[:5])
        assert has(r, "t3", m[:3]) and has(r, "t3", m[2:5])
        assert has(r, "t5", m) == present
        mask, _, _ = _t5(ora_barrel, e2, d[:5])
        assert mask == (ALL_T5 if present else ALL_T5 & ~T5_BRFULL)


def test_t5_full_radius_threshold(barrel_geom, ora_barrel):
    """The full circle needs R >= 0.95 Rmin (0.76 GeV): the five anchors of a 0.72 GeV helix
    fail only that condition, those of a 0.78 GeV helix pass all four."""
    for pt, ok in ((0.72, False), (0.78, True)):
        ev = event(barrel_geom, track(pt, 0.4, 0.1))
        d = doublets(ev)
        assert len(d) >= 5
        mask, _, kf = _t5(ora_barrel, ev, d[:5])
        assert mask == (ALL_T5 if ok else ALL_T5 & ~T5_RADIUS)
        assert abs(1 / abs(kf) - pt / 0.0113922) / (pt / 0.0113922) < 2e-3


def test_t5_rz_rejects_kink(barrel_geom, ora_barrel):
    """A kink in r-z at the shared MD c: a, b, c on one straight line and c, d, e on another
    (both T3s straight), so only (a, c, e) is not straight.  A slope change of 0.10 (e moves
    5.9 cm in z) is beyond the hits' z tolerance (PS/2S resolution over the lever arms) and
    removes T5 (1..5) with only the r-z condition failing; 0.01 keeps it."""
    t, ev, d = _t5_case(barrel_geom)
    P = points(ev)
    rc = np.hypot(*P[d[2][1], :2])
    for slope, present in ((0.10, False), (0.01, True)):
        ch = {}
        for x in d[3:5]:
            for h in (x[1], x[2]):
                s = np.hypot(*P[h, :2]) - rc  # transverse distance beyond c (stiff track)
                ch[h] = (P[h, 0], P[h, 1], P[h, 2] + slope * s)
        e2 = edited(ev, ch)
        r = oracle.run(ora_barrel, e2)
        m = _mds(r, d[:5])
        assert has(r, "t3", m[:3]) and has(r, "t3", m[2:5])
        assert has(r, "t5", m) == present
        mask, _, _ = _t5(ora_barrel, e2, d[:5])
        assert mask == (ALL_T5 if present else ALL_T5 & ~T5_RZ)


# ---------------------------------------------------------------- pLS anchors, pT5 curvature
def _seeded(barrel_geom, pt):
    for phi0 in np.linspace(0.11, 6.1, 41):
        ev = event(barrel_geom, track(pt, phi0, 0.2), pls=True)
        d = doublets(ev)
        if len(d) == 6 and ev.n_pls == 1:
            return ev, d
    raise AssertionError


def test_pls_window_rejects_rotated_seed(barrel_geom, ora_barrel):
    """A seed direction off by theta moves the extrapolated circle by about theta x s at arc
    length s; the r-phi window grows as 0.02 cm + 3 mrad x s (+ the curvature term), about
    4.7 mrad x s at the first outer layer.  Rotated by 6.5 mrad the seed links to nothing
    (r-phi fails, r-z passes: the pLS stays a candidate on its own); by 1 mrad it forms its pT5."""
    ev, d = _seeded(barrel_geom, 5.0)
    for theta, linked in ((6.5e-3, False), (1.0e-3, True)):
        pls = ev.pls.copy()
        c, s = np.cos(theta), np.sin(theta)
        px, py = float(pls["px"][0]), float(pls["py"][0])
        pls["px"][0], pls["py"][0] = px * c - py * s, px * s + py * c
        e2 = edited(ev, {}, pls=pls)
        r = oracle.run(ora_barrel, e2)
        assert (len(r["pt5"]) > 0) == linked and (len(r["pt3"]) > 0) == linked
        assert bool(r["pls_tc"][0]) == (not linked)
        mask, _ = oracle.pls_eval(ora_barrel, pls[0], d[0][0], points(e2)[d[0][1]])
        assert mask == (PLS_RPHI | PLS_RZ if linked else PLS_RZ)


def test_pt5_curvature_rejects_wrong_seed_pt(barrel_geom, ora_barrel):
    """A pT5 needs the T5's curvature within 15 % of the seed's.  A 50 GeV track whose seed
    claims 1.3 x its pT keeps its pT3 (the anchor windows still hold at this stiffness) but
    forms no pT5, with only the curvature condition failing; a seed at 1.1 x forms it."""
    ev, d = _seeded(barrel_geom, 50.0)
    for scale, ok in ((1.3, False), (1.1, True)):
        pls = ev.pls.copy()
        for k in ("px", "py", "pz"):
            pls[k][0] = pls[k][0] * scale
        e2 = edited(ev, {}, pls=pls)
        r = oracle.run(ora_barrel, e2)
        assert len(r["pt3"]) > 0
        assert (len(r["pt5"]) > 0) == ok
        P = points(e2)
        mask = oracle.pt5_eval(ora_barrel, pls[0], [x[0] for x in d[:5]], [P[x[1]] for x in d[:5]])
        assert mask == (PT5_WINDOWS | PT5_CURV if ok else PT5_WINDOWS)


# ---------------------------------------------------------------- pins found by planted mistakes
def test_endcap_doublets_with_resolution(full_geom, ora_full):
    """Endcap sensors measure r to 0.5 mm: the hit-pair windows widen by that (radial
    tolerance in the bending slope, its offset across the step, and the r-z pointing),
    so >= 95 % of reachable true endcap MDs and >= 90 % of true disk-to-disk LSs survive."""
    import lst_synth as S
    from lst_synth import events as E
    rng = np.random.default_rng(51)
    t = E.random_tracks(rng, 400, pt_mode="uniform", pt_lo=1.0, pt_hi=10.0, eta_max=2.4)
    t["eta"] = np.sign(t["eta"]) * (1.7 + np.abs(t["eta"]) * (0.7 / 2.4))
    ev = E.event_from_tracks(full_geom, t, 51, exact=False)
    r = oracle.run(ora_full, ev)
    mods = full_geom.modules
    md = r["md"]
    endcap = mods["subdet"][md[:, 0]] == 1
    true_md = ev.sim[md[:, 1]] == ev.sim[md[:, 2]]
    m_ec = (mods["subdet"][ev.det >> 1] == 1)
    key = ev.sim.astype(np.int64) * 100000 + (ev.det >> 1)
    u, c = np.unique(key[m_ec], return_counts=True)
    reachable = int((c == 2).sum())
    assert reachable > 1000
    assert (true_md & endcap).sum() >= 0.95 * reachable
    # true LSs between consecutive disks of one track
    ls = r["ls"]
    a, b = md[ls[:, 0]], md[ls[:, 1]]
    same = (ev.sim[a[:, 1]] == ev.sim[b[:, 1]]) & (ev.sim[a[:, 1]] >= 0)
    disk_pair = (mods["subdet"][a[:, 0]] == 1) & (mods["subdet"][b[:, 0]] == 1)
    got = {(int(ev.sim[x[1]]), int(mods["layer"][x[0]])) for x in a[same & disk_pair]}
    trk_md = {}
    for k in np.nonzero(true_md & endcap)[0]:
        trk_md.setdefault(int(ev.sim[md[k, 1]]), set()).add(int(mods["layer"][md[k, 0]]))
    want = {(s, d) for s, ds in trk_md.items() for d in ds if d + 1 in ds}
    assert len(want) > 500 and len(got & want) >= 0.9 * len(want)


def test_bending_rejects_backward_step(full_geom, ora_full):
    """A track leaving the beam line moves outward: a disk-to-disk pair whose outer hit
    lies radially inward of the inner one, beyond the two hits' radial tolerance, fails the
    bending condition even with no sideways offset; the same step outward passes it."""
    mods = full_geom.modules
    A = int(np.nonzero((mods["subdet"] == 1) & (mods["side"] == 1) & (mods["layer"] == 1) & (mods["ieta"] == 3))[0][0])
    B = int(np.nonzero((mods["subdet"] == 1) & (mods["side"] == 1) & (mods["layer"] == 2) & (mods["ieta"] == 3)
                       & (mods["iphi"] == mods["iphi"][A]))[0][0])
    phi = 0.5 * (np.arctan2(mods["e0y"][A], mods["e0x"][A]) + np.arctan2(mods["e1y"][A], mods["e1x"][A]))
    u = np.array([np.cos(phi), np.sin(phi)])
    ra = 55.0
    za, zb = float(mods["surf"][A]), float(mods["surf"][B])
    for step, ok in ((-0.33, False), (0.33, True)):
        a = (*(ra * u), za)
        b = (*((ra + step) * u), zb)
        mask = oracle.ls_eval(ora_full, A, B, a, (a[0], a[1], za + 0.4), b, (b[0], b[1], zb + 0.4))
        assert bool(mask & LS_BEND) == ok


@pytest.mark.parametrize("side", [1, -1])
def test_ls_barrel_exit_both_sides(full_geom, ora_full, side):
    """The barrel exit (|z| = 120) holds on both ends of the barrel."""
    mods = full_geom.modules
    for cot, present in ((1.36, False), (1.40, True)):
        eta = side * np.arcsinh(cot)
        for phi0 in np.linspace(0.13, 6.1, 37):
            ev = event(full_geom, track(10.0, phi0, eta, -1))
            d = doublets(ev)
            l4 = [x for x in d if mods[x[0]]["subdet"] == 0 and mods[x[0]]["layer"] == 4]
            d1 = [x for x in d if mods[x[0]]["subdet"] == 1 and mods[x[0]]["layer"] == 1]
            if l4 and d1:
                break
        r = oracle.run(ora_full, ev)
        m = _mds(r, (l4[0], d1[0]))
        assert m[0] is not None and m[1] is not None
        assert has(r, "ls", m) == present
        assert _ls_mask(ora_full, ev, l4[0], d1[0]) == (ALL_LS if present else ALL_LS & ~LS_EXIT)


def test_t5_radius_condition_is_on_the_full_circle(barrel_geom, ora_barrel):
    """The radius condition belongs to the (a, c, e) circle: five anchors whose inner
    triple is stiffer than the 0.76 GeV limit but whose full circle is not fail it, and the
    reverse passes it (only that bit is read here)."""
    from scipy.optimize import brentq
    kmax = 1.0 / (0.95 * RMIN)
    for pt_in, pt_full, ok in ((0.9, 0.70, False), (0.70, 0.9, True)):
        ev = event(barrel_geom, track(pt_full, 0.4, 0.1))
        d = doublets(ev)
        P = points(ev)
        t = track(pt_full, 0.4, 0.1)
        A = [P[x[1], :2] for x in d[:5]]
        nb = outward(t, A[1])
        # move b across the track until the inner triple has the curvature of pt_in
        k_target = np.sign(curvature(A[0], A[1], A[2])) * 0.0113922 / pt_in
        eb = brentq(lambda x: curvature(A[0], A[1] + x * nb, A[2]) - k_target, -5.0, 5.0)
        e2 = edited(ev, shift_doublet(ev, d[1], dxy=eb * nb))
        mask, _, kf = _t5(ora_barrel, e2, d[:5])
        assert (abs(kf) > kmax) != ok
        assert bool(mask & T5_RADIUS) == ok


def test_t5_score_sums_both_disagreements(barrel_geom, ora_barrel):
    """The T5 score is the inner/outer plus the bridge/full curvature disagreement: a
    construction that moves only the bridge curvature gives a score equal to that
    disagreement, one that moves only the inner/outer pair gives that one."""
    t, ev, d = _t5_case(barrel_geom)
    P = points(ev)
    A = [P[x[1], :2] for x in d[:5]]
    nb, nd = outward(t, A[1]), outward(t, A[3])
    # b and d outward by amounts giving equal inner and outer curvature changes
    eb = 0.05
    dk = curvature(A[0], A[1] + eb * nb, A[2]) - curvature(A[0], A[1], A[2])
    from scipy.optimize import brentq
    ed = brentq(lambda x: curvature(A[2], A[3] + x * nd, A[4]) - curvature(A[2], A[3], A[4]) - dk, -5, 5)
    ch = shift_doublet(ev, d[1], dxy=eb * nb)
    ch.update(shift_doublet(ev, d[3], dxy=ed * nd))
    e2 = edited(ev, ch)
    Q = [points(e2)[x[1], :2] for x in d[:5]]
    dbr = abs(curvature(Q[1], Q[2], Q[3]) - curvature(Q[0], Q[2], Q[4]))
    dio = abs(curvature(Q[0], Q[1], Q[2]) - curvature(Q[2], Q[3], Q[4]))
    _, score, _ = _t5(ora_barrel, e2, d[:5])
    assert dbr > 20 * dio
    assert abs(float(score) - (dbr + dio)) <= 1e-3 * dbr + 2e-7


def test_pls_window_allows_seed_curvature_error(barrel_geom, ora_barrel):
    """Seeds carry a 1 % pT error; the r-phi window grows with the curvature error's
    sagitta (1.5 % x s^2 / R, three sigma of half the relative error).  A 0.9 GeV track whose
    seed is off by +2.5 % in pT still forms its pT5 over five layers; off by +6 % it does not
    (the outer anchors leave the window), though its direction and dip are exact."""
    ev, d = _seeded(barrel_geom, 0.9)
    for scale, linked in ((1.025, True), (1.06, False)):
        pls = ev.pls.copy()
        for k in ("px", "py", "pz"):
            pls[k][0] = pls[k][0] * scale
        r = oracle.run(ora_barrel, edited(ev, {}, pls=pls))
        assert (len(r["pt5"]) > 0) == linked


def test_pls_window_rejects_wrong_dip(barrel_geom, ora_barrel):
    """A seed whose dip (cot theta) is off by 0.02 misses the first anchor's r-z window
    (0.4 cm off at 20 cm against 0.05 cm + 2 mrad x s + the PS z resolution): no pT3 and
    only the r-z window fails there; off by 0.002 it links."""
    ev, d = _seeded(barrel_geom, 5.0)
    for dcot, linked in ((0.02, False), (0.002, True)):
        pls = ev.pls.copy()
        pt = float(np.hypot(pls["px"][0], pls["py"][0]))
        pls["pz"][0] = pls["pz"][0] + dcot * pt
        e2 = edited(ev, {}, pls=pls)
        r = oracle.run(ora_barrel, e2)
        assert (len(r["pt3"]) > 0) == linked
        mask, _ = oracle.pls_eval(ora_barrel, pls[0], d[0][0], points(e2)[d[0][1]])
        assert mask == (PLS_RPHI | PLS_RZ if linked else PLS_RPHI)


def test_tracks_sharing_two_doublets_stay_two_candidates(barrel_geom, ora_barrel):
    """Duplicates are the same particle found twice and share most of their MDs (3 of 5
    for pT5s and T5s); two particles that only cross the first two layers at the same
    points are two tracks.  Track B is built through track A's layer-1 and layer-2 anchors
    with another radius (a 0.4 cm impact parameter); with exact seeds for both, the
    candidates are A's pT5 and B's pT5."""
    from lst_synth import events as E
    ta, ev, d = clean_track(barrel_geom, 5.0, 0.2, 6)
    P = points(ev)
    _, _, cx, cy = E.helix_centre(ta)
    tb = track_through(P[d[0][1]], P[d[1][1]], 300.0, int(ta["q"][0]), 0.2, np.array([cx[0], cy[0]]))
    evb = event(barrel_geom, tb)
    db = doublets(evb)
    assert len(db) == 6
    # B's own hits from layer 3 on, A's doublets on layers 1 and 2
    keep = np.concatenate([[x[1], x[2]] for x in db[2:]])
    t2 = np.concatenate([ta, tb])
    rng = np.random.default_rng(0)
    pls, pls_sim = E.make_pls(rng, t2, np.array([0, 1]), 0, exact=True)
    both = E.Event(np.concatenate([ev.x, evb.x[keep]]), np.concatenate([ev.y, evb.y[keep]]),
                   np.concatenate([ev.z, evb.z[keep]]), np.concatenate([ev.det, evb.det[keep]]),
                   np.concatenate([ev.sim, np.ones(len(keep), np.int32)]), t2, pls, pls_sim)
    r = oracle.run(ora_barrel, both)
    mdA = _mds(r, d[:5])
    dB = [d[0], d[1]] + [(x[0], ev.n_hits + 2 * (k - 2), ev.n_hits + 2 * (k - 2) + 1) for k, x in enumerate(db) if k >= 2]
    mdB = _mds(r, dB[:5])
    assert None not in mdA and None not in mdB
    t5 = [tuple(map(int, x)) for x in r["t5"]]
    assert tuple(mdA) in t5 and tuple(mdB) in t5
    assert sorted(r["tc_type"].tolist()) == [0, 0]
    assert sorted(r["tc_pls"].tolist()) == [0, 1]
    assert sorted(r["tc_pt"].tolist()) == pytest.approx(sorted([5.0, 300.0 * 0.0113922]), rel=1e-4)


def test_t5_candidate_pt_is_the_helix_pt(barrel_geom, ora_barrel):
    """A T5 candidate's pT is the field constant over its full-circle curvature,
    pT = 0.3 B R (R in m): on noiseless 1-20 GeV tracks it equals the simulated pT."""
    from lst_synth import events as E
    rng = np.random.default_rng(61)
    t = E.random_tracks(rng, 30, pt_mode="uniform", pt_lo=1.0, pt_hi=20.0, eta_max=0.8)
    n = 0
    for i in range(len(t)):
        ev = event(barrel_geom, t[i:i + 1])
        if len(doublets(ev)) != 6:
            continue
        r = oracle.run(ora_barrel, ev)
        assert list(r["tc_type"]) == [2]
        assert abs(r["tc_pt"][0] - t["pt"][i]) / t["pt"][i] < 2e-3
        n += 1
    assert n > 15


def test_pt3_sharing_two_mds_with_a_pt5_is_removed(barrel_geom, ora_barrel):
    """Across stages a pT3 that shares two of its three MDs with a surviving pT5 is a
    duplicate of it.  Track B (50 GeV) passes through track A's (5 GeV) layer-2 and layer-3
    anchors, which every T5 of A contains; A's exact seed forms A's pT5; B's seed, whose pT
    is 1.3 x too high, forms only pT3s, each on (b1, a2, a3) or (a2, a3, b4), which must go:
    B's seed stays a pLS candidate and no pT3 candidate comes out."""
    from lst_synth import events as E
    ta, ev, d = clean_track(barrel_geom, 5.0, 0.2, 6)
    P = points(ev)
    _, _, cx, cy = E.helix_centre(ta)
    tb = track_through(P[d[1][1]], P[d[2][1]], 50.0 / 0.0113922, int(ta["q"][0]), 0.2, np.array([cx[0], cy[0]]))
    evb = event(barrel_geom, tb)
    db = doublets(evb)
    assert len(db) == 6
    keep = np.concatenate([[x[1], x[2]] for k, x in enumerate(db) if k not in (1, 2)])
    t2 = np.concatenate([ta, tb])
    pls, pls_sim = E.make_pls(np.random.default_rng(0), t2, np.array([0, 1]), 0, exact=True)
    for k in ("px", "py", "pz"):
        pls[k][1] = pls[k][1] * 1.3
    both = E.Event(np.concatenate([ev.x, evb.x[keep]]), np.concatenate([ev.y, evb.y[keep]]),
                   np.concatenate([ev.z, evb.z[keep]]), np.concatenate([ev.det, evb.det[keep]]),
                   np.concatenate([ev.sim, np.ones(len(keep), np.int32)]), t2, pls, pls_sim)
    r = oracle.run(ora_barrel, both)
    mA = _mds(r, d)
    # B's seed built pT3s only, each sharing A's layer-2 and layer-3 MDs
    t3 = r["t3"]
    pt3_b = np.nonzero(r["pt3"][:, 0] == 1)[0]
    assert len(pt3_b) >= 1 and not np.any(r["pt5"][:, 0] == 1)
    for k in pt3_b:
        assert len({mA[1], mA[2]} & set(t3[r["pt3"][k, 1]].tolist())) == 2
    alive5 = r["pt5"][r["alive_pt5"] == 1]
    assert len(alive5) == 1 and alive5[0, 0] == 0
    assert not np.any(r["alive_pt3"][pt3_b])
    types = sorted(zip(r["tc_type"].tolist(), r["tc_pls"].tolist()))
    assert (0, 0) in types and (3, 1) in types and all(t != 1 for t, _ in types)


def test_triplet_seeds_link_like_quads(barrel_geom, ora_barrel):
    """A pixel triplet (one of the four pixel hits missing, Sec. 2: legacy and LST
    triplets) carries the same helix at its first remaining hit: exact triplet seeds of
    clean tracks form the same pT5 as the quad would, with the three pixel hits in the
    candidate; with the first hit missing, the reference point moves to the second pixel
    layer and the seed still links."""
    from lst_synth import events as E
    n = 0
    for phi0 in np.linspace(0.3, 6.0, 12):
        t = track(4.0, phi0, 0.2)
        ev = E.event_from_tracks(barrel_geom, t, 5, exact=True, with_pls=True, fake_pls_frac=0.0, shuffle=False)
        if len(doublets(ev)) != 6 or ev.n_pls != 1:
            continue
        quad = oracle.run(ora_barrel, ev)
        assert list(quad["tc_type"]) == [0]
        for drop in (0, 2):
            pls, _ = E.make_pls(np.random.default_rng(0), t, np.array([0]), 0, exact=True)
            keep = [k for k in range(4) if k != drop]
            for key in ("hx", "hy", "hz"):
                pls[key][0] = np.concatenate([pls[key][0][keep], [0.0]])
            pls["n_hits"][0] = 3
            if drop == 0:
                a = E.cylinder_alpha(t, E.PIXEL_R[1])
                x, y, z, ph = E.helix_point(t, a)
                pls["x0"][0], pls["y0"][0], pls["z0"][0] = x[0], y[0], z[0]
                ptr = float(np.hypot(pls["px"][0], pls["py"][0]))
                pls["px"][0], pls["py"][0] = ptr * np.cos(ph[0]), ptr * np.sin(ph[0])
            r = oracle.run(ora_barrel, edited(ev, {}, pls=pls))
            assert list(r["tc_type"]) == [0]
            assert list(r["tc_pix"][0]) == [0, 1, 2, 0xFFFFFFFF]
            assert r["tc_pt"][0] == pytest.approx(4.0, rel=1e-5)
            n += 1
    assert n >= 10
