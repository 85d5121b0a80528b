"""Pins of the oracle on the geometry whose outer endcap rings are 2S modules (Fig. 1).

In that geometry the disk rings starting at r >= 60 cm are strip-strip modules: a hit
there measures the azimuth, and its radius only as the centre of a 5 cm radial strip, so
the module's radial tolerance is half a strip plus 0.5 mm.  The cut forms are those of the
PS endcap with that tolerance in place.  These pins check that the synthetic readout is
what that reading assumes, that true doublets and disk-to-disk segments through 2S rings
survive it, that the connection map loses no LS, and that the joins equal brute force.
"""
import numpy as np

import lst_synth as S
import oracle
from lst_synth import events as E
GM = E.G  # the geometry module (the package exports a function of that name)


def _forward_tracks(seed, n):
    rng = np.random.default_rng(seed)
    t = E.random_tracks(rng, n, pt_mode="uniform", pt_lo=1.0, pt_hi=10.0, eta_max=2.4)
    t["eta"] = np.sign(t["eta"]) * (1.5 + np.abs(t["eta"]) * (0.9 / 2.4))
    return t


def test_2s_ring_hits_read_the_strip_centre(ec2s_geom):
    """A hit on a 2S endcap module has r = inner edge + (k + 1/2) x 5 cm and keeps the
    azimuth of the crossing to the r-phi resolution; PS rings keep r to 0.5 mm."""
    t = _forward_tracks(61, 300)
    ev = E.event_from_tracks(ec2s_geom, t, 61, noise_frac=0.0, exact=False, shuffle=False)
    ex = E.event_from_tracks(ec2s_geom, t, 61, noise_frac=0.0, exact=True, shuffle=False)
    mods = ec2s_geom.modules
    m = mods[ev.det >> 1]
    ring_2s = (m["subdet"] == 1) & (m["stype"] == GM.STYPE_2S)
    ring_ps = (m["subdet"] == 1) & (m["stype"] == GM.STYPE_PS)
    assert ring_2s.sum() > 500 and ring_ps.sum() > 500
    # the same crossings in the same order with and without the readout model
    assert np.array_equal(ev.det, ex.det) and np.array_equal(ev.sim, ex.sim)
    r = np.hypot(ev.x.astype(np.float64), ev.y.astype(np.float64))
    r_true = np.hypot(ex.x.astype(np.float64), ex.y.astype(np.float64))
    k = (r[ring_2s] - m["emin"][ring_2s]) / 5.0 - 0.5
    assert np.all(np.abs(k - np.round(k)) < 1e-4)
    assert np.all(np.abs(r[ring_2s] - r_true[ring_2s]) <= 2.5 + 1e-4)
    assert np.all(m["emin"][ring_2s] >= GM.RING_2S_R - 1e-3)
    assert np.all(np.abs(r[ring_ps] - r_true[ring_ps]) < 0.5)
    dphi = np.angle(np.exp(1j * (np.arctan2(ev.y, ev.x) - np.arctan2(ex.y, ex.x))))
    assert np.all(np.abs(dphi * r_true)[ring_2s] < 6 * 0.003)  # 30 um r-phi, 6 sigma
    assert np.array_equal(ev.z[m["subdet"] == 1], ex.z[m["subdet"] == 1])  # disks: z is the sensor plane


def test_2s_ring_doublets_and_segments_with_resolution(ec2s_geom, ora_ec2s):
    """With the 2S readout, the half-strip radial tolerance keeps the true doublets on 2S
    rings and the true segments between consecutive disks that end on a 2S ring (>= 99.5 %
    and >= 99 %; all of them in this sample; with the PS rings' 0.15 cm tolerance 2 % of
    the doublets and 6 % of the segments are lost)."""
    t = _forward_tracks(62, 400)
    ev = E.event_from_tracks(ec2s_geom, t, 62, exact=False)
    r = oracle.run(ora_ec2s, ev)
    mods = ec2s_geom.modules
    md = r["md"]
    ring_2s_md = (mods["subdet"][md[:, 0]] == 1) & (mods["stype"][md[:, 0]] == GM.STYPE_2S)
    true_md = ev.sim[md[:, 1]] == ev.sim[md[:, 2]]
    on_2s = (mods["subdet"][ev.det >> 1] == 1) & (mods["stype"][ev.det >> 1] == GM.STYPE_2S)
    key = ev.sim.astype(np.int64) * 100000 + (ev.det >> 1)
    _, c = np.unique(key[on_2s], return_counts=True)
    reachable = int((c == 2).sum())
    assert reachable > 300
    assert (true_md & ring_2s_md).sum() >= 0.995 * reachable
    ls = r["ls"]
    a, b = md[ls[:, 0]], md[ls[:, 1]]
    same = (ev.sim[a[:, 1]] == ev.sim[b[:, 1]]) & (ev.sim[a[:, 1]] >= 0)
    disks = (mods["subdet"][a[:, 0]] == 1) & (mods["subdet"][b[:, 0]] == 1)
    got = {(int(ev.sim[x[1]]), int(mods["layer"][x[0]])) for x in a[same & disks]}
    trk = {}
    for k in np.nonzero(true_md & (mods["subdet"][md[:, 0]] == 1))[0]:
        trk.setdefault(int(ev.sim[md[k, 1]]), {})[int(mods["layer"][md[k, 0]])] = int(md[k, 0])
    want = {(s, d) for s, ds in trk.items() for d in ds
            if d + 1 in ds and mods["stype"][ds[d + 1]] == GM.STYPE_2S}
    assert len(want) > 100 and len(got & want) >= 0.99 * len(want)


def test_2s_connection_map_loses_no_ls(ora_ec2s):
    """The map's bound carries the 2S rings' radial tolerance: no LS is lost against
    testing every MD pair on adjacent surfaces."""
    for n, i in ((300, 1), (700, 2)):
        ev = S.make_event("pu200", i, n_tracks=n, endcap_2s=True)
        a = oracle.run(ora_ec2s, ev)
        b = oracle.run(ora_ec2s, ev, brute_ls=True)
        assert len(a["ls"]) > 0
        assert np.array_equal(a["ls"], b["ls"]) and np.array_equal(a["t5"], b["t5"])
