"""Brute-force enumerations against the oracle's joins.

The chain builds objects by walking lists (connection map, per-MD LS/T3/T5 offsets, pLS
candidate modules).  Here every combination is enumerated in Python on small events and
decided by the predicate-level evaluation alone: all MD pairs on adjacent surfaces (LS),
all MD triples (T3), all 5-chains (T5), every pLS against every T3/T5 that starts on a
surface the pLS lookup covers, with no module filter (pT3/pT5).  The object sets, their
order and their float results must equal the chain's.  A wrong offset, index or loop bound
in a join, a module missing from the map or from a pLS's candidates, or a score summed in
another order fails here.  A separate test checks the pLS candidate modules against the
helix crossing computed in float64 by the input generator's own helix code.
"""
import numpy as np
import pytest

import lst_synth as S
import oracle
from lst_synth import events as E
G = E.G  # the detector-description module (lst_synth.geometry)

ALL_LS, ALL_T3, ALL_T5 = 31, 7, 15


def surface(m):
    """0..5 barrel layers, 6..10 disks z < 0, 11..15 disks z > 0."""
    if m["subdet"] == 0:
        return int(m["layer"]) - 1
    return (6 if m["side"] < 0 else 11) + int(m["layer"]) - 1


def next_surfaces(s):
    """Surfaces a track leaving surface s can cross next (barrel layer -> next layer or
    first disk of either side; disk -> next disk on the same side)."""
    if s < 6:
        return ([s + 1] if s < 5 else []) + [6, 11]
    if s < 11:
        return [s + 1] if s < 10 else []
    return [s + 1] if s < 15 else []


def _brute(geom, og, ev):
    r = oracle.run(og, ev)
    mods = geom.modules
    md = r["md"]
    P = np.stack([ev.x, ev.y, ev.z], 1)
    surf = np.array([surface(mods[m]) for m in md[:, 0]], np.int64)
    by_surf = {s: np.nonzero(surf == s)[0] for s in range(16)}
    ls = []
    for i in range(len(md)):
        for s in next_surfaces(int(surf[i])):
            for j in by_surf[s]:
                m = oracle.ls_eval(og, int(md[i, 0]), int(md[j, 0]), P[md[i, 1]], P[md[i, 2]], P[md[j, 1]], P[md[j, 2]])
                if m == ALL_LS:
                    ls.append((i, int(j)))
    ls.sort()
    out = {}
    for a, b in ls:
        out.setdefault(a, []).append(b)
    t3 = []
    for a, b in ls:
        for c in out.get(b, []):
            m = oracle.t3_eval(og, (md[a, 0], md[b, 0], md[c, 0]), P[md[a, 1]], P[md[b, 1]], P[md[b, 2]], P[md[c, 1]])
            if m == ALL_T3:
                t3.append((a, b, c))
    t3.sort()
    t3_from = {}
    for t in t3:
        t3_from.setdefault(t[0], []).append(t)
    t5, score, kfull = [], [], []
    for t in t3:
        for u in t3_from.get(t[2], []):
            ch = t + u[1:]
            m, sc, kf = oracle.t5_eval(og, md[list(ch), 0], P[md[list(ch), 1]])
            if m == ALL_T5:
                t5.append(ch)
                score.append(sc)
                kfull.append(kf)
    idx = sorted(range(len(t5)), key=lambda k: t5[k])
    return r, ls, t3, [t5[k] for k in idx], np.array([score[k] for k in idx], np.float32), \
        np.array([kfull[k] for k in idx], np.float32)


@pytest.mark.parametrize("case", ["tiny", "barrel_res", "pu200_small", "tilted_small", "endcap_2s_small",
                                  "pu200_learned_t5"])
def test_ls_t3_t5_equal_brute_force(case, barrel_geom, full_geom, ora_barrel, ora_full, tilted_geom, ora_tilted,
                                    ec2s_geom, ora_ec2s):
    if case == "endcap_2s_small":
        geom, og = ec2s_geom, ora_ec2s
        ev = S.make_event("pu200", 9, n_tracks=80, endcap_2s=True)
    elif case == "pu200_learned_t5":  # the T5 step with the shipped network in place of the kappa cuts
        import paper_2407_18231_gb300 as lst
        geom, og = full_geom, oracle.Geometry(full_geom.modules)
        oracle.set_t5_mlp(og, lst.load_t5_mlp())
        ev = S.make_event("pu200", 5, n_tracks=50)
    elif case == "tilted_small":
        geom, og = tilted_geom, ora_tilted
        ev = S.make_event("pu200", 8, n_tracks=60, realistic=True)
    elif case == "tiny":
        geom, og, ev = barrel_geom, ora_barrel, S.make_event("tiny")
    elif case == "barrel_res":
        geom, og = barrel_geom, ora_barrel
        ev = S.make_event("batched", 3, n_tracks=25)
    else:
        geom, og = full_geom, ora_full
        ev = S.make_event("pu200", 5, n_tracks=50)
    r, ls, t3, t5, score, kfull = _brute(geom, og, ev)
    assert len(t5) > 0
    assert [tuple(map(int, x)) for x in r["ls"]] == ls
    assert [tuple(map(int, x)) for x in r["t3"]] == t3
    assert [tuple(map(int, x)) for x in r["t5"]] == t5
    assert r["t5_score"].tobytes() == score.tobytes()
    assert r["t5_kfull"].tobytes() == kfull.tobytes()


def _pls_surfaces(geom):
    """Surfaces the pLS lookup covers: barrel layers 1-2 and the first two disks."""
    return {0, 1, 6, 7, 11, 12}


@pytest.mark.parametrize("exact", [True, False])
def test_pt3_pt5_equal_brute_force_without_module_filter(exact, full_geom, ora_full):
    ev = S.make_event("pu200", 6, n_tracks=60, with_pls=True, exact=exact)
    r = oracle.run(ora_full, ev)
    mods = full_geom.modules
    md = r["md"]
    P = np.stack([ev.x, ev.y, ev.z], 1)
    cover = _pls_surfaces(full_geom)
    starts = {i for i in range(len(md)) if surface(mods[md[i, 0]]) in cover}
    assert len(r["pt3"]) > 0 and len(r["pt5"]) > 0
    memo = {}

    def anchor(p, m):
        if (p, m) not in memo:
            memo[(p, m)] = oracle.pls_eval(ora_full, ev.pls[p], int(md[m, 0]), P[md[m, 1]])
        return memo[(p, m)]

    pt3, pt3_score = [], []
    for p in range(ev.n_pls):
        for t, obj in enumerate(r["t3"]):
            if int(obj[0]) not in starts:
                continue
            res = [anchor(p, int(m)) for m in obj]
            if all(x[0] == 3 for x in res):
                sc = np.float32(0)
                for _, s in res:
                    sc = np.float32(sc + s)
                pt3.append((p, t))
                pt3_score.append(sc)
    assert [tuple(map(int, x)) for x in r["pt3"]] == pt3
    assert r["pt3_score"].tobytes() == np.array(pt3_score, np.float32).tobytes()
    pt5 = []
    for p in range(ev.n_pls):
        for t, obj in enumerate(r["t5"]):
            if int(obj[0]) not in starts:
                continue
            if oracle.pt5_eval(ora_full, ev.pls[p], md[obj, 0], P[md[obj, 1]]) == 3:
                pt5.append((p, t))
    assert [tuple(map(int, x)) for x in r["pt5"]] == pt5


def _seed_tracks(ev):
    """The seeds' own helices as generator tracks (float64)."""
    t = np.zeros(ev.n_pls, E.TRACK_DTYPE)
    s = ev.pls
    pt = np.hypot(s["px"].astype(np.float64), s["py"].astype(np.float64))
    t["pt"] = pt
    t["phi0"] = np.arctan2(s["py"].astype(np.float64), s["px"].astype(np.float64))
    t["eta"] = np.arcsinh(s["pz"].astype(np.float64) / pt)
    t["q"] = s["charge"]
    t["vx"], t["vy"], t["vz"] = s["x0"], s["y0"], s["z0"]
    return t


@pytest.mark.parametrize("exact", [True, False])
def test_pls_candidates_around_float64_crossings(exact, full_geom, ora_full):
    """Each seed's candidate list holds the module that contains the helix crossing of
    barrel layers 1-2 and of the first two disks on its pz side (crossing computed in
    float64 by the generator's helix code); where a crossing is clear of module edges its
    whole neighbourhood (+-1 row, +-1 sector) is listed; and no candidate lies farther from
    every crossing than one row and one sector (two next to an edge, where float32 and
    float64 may pick neighbouring cells)."""
    ev = S.make_event("pu200", 7, n_tracks=300, with_pls=True, exact=exact)
    r = oracle.run(ora_full, ev)
    geom = full_geom
    mods = geom.modules
    t = _seed_tracks(ev)
    n_checked = n_clear = 0
    for p in range(ev.n_pls):
        cand = set(r["pls_cand"][p][: r["pls_cand_n"][p]].tolist())
        tp = t[p:p + 1]
        allowed = set()
        for kind, layer in (("b", 1), ("b", 2), ("e", 1), ("e", 2)):
            side = 0
            if kind == "b":
                a = E.cylinder_alpha(tp, G.BARREL_R[layer - 1])
            else:
                side = 1 if tp["eta"][0] > 0 else -1
                a = E.plane_alpha(tp, side * G.DISK_Z[layer - 1])
            if np.isnan(a[0]):
                continue
            x, y, z, _ = E.helix_point(tp, a)
            x, y, z = float(x[0]), float(y[0]), float(z[0])
            phi = np.arctan2(y, x) % (2 * np.pi)
            if kind == "b":
                u, nrow = (z + G.BARREL_ZHALF) / G.BARREL_ZLEN, G.BARREL_NZ
                m0 = int(geom.barrel_module(np.array([layer]), np.array([z]), np.array([phi]))[0])
            else:
                rr = np.hypot(x, y)
                u, nrow = (rr - G.RING_R0) / G.RING_DR, G.N_RING
                m0 = int(geom.endcap_module(np.array([side]), np.array([layer]), np.array([rr]), np.array([phi]))[0])
            if m0 >= 0:
                n_checked += 1
                assert m0 in cand, (p, kind, layer)
            row = int(np.floor(u))
            near_row = not 0.02 < u - row < 0.98
            for rw in range(row - 2, row + 3):
                if not 0 <= rw < nrow or (abs(rw - row) == 2 and not near_row):
                    continue
                nphi = geom.barrel_nphi[layer - 1] if kind == "b" else geom.ring_nphi[rw]
                base = (geom.barrel_base[layer - 1] + rw * nphi) if kind == "b" else geom.endcap_base[(side, layer)][rw]
                v = phi / (2 * np.pi / nphi)
                sec = int(np.floor(v)) % nphi
                near_sec = not 0.02 < v - np.floor(v) < 0.98
                reach = 2 if (near_sec or kind == "e") else 1
                for ds in range(-reach, reach + 1):
                    allowed.add(base + (sec + ds) % nphi)
                same_ring = kind == "b" or geom.ring_nphi[rw] == geom.ring_nphi[min(max(row, 0), nrow - 1)]
                if abs(rw - row) <= 1 and not near_row and not near_sec and same_ring and 0 <= row < nrow:
                    n_clear += 1
                    for ds in (-1, 0, 1):
                        assert base + (sec + ds) % nphi in cand, (p, kind, layer, rw, ds)
        assert cand <= allowed, (p, sorted(cand - allowed))
    assert n_checked > 300 and n_clear > 300
