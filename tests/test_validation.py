"""Track-level metrics (Sec. 3): the hit-match rule, efficiency, fake and duplicate rates.

Hand-built candidates pin the definitions (strictly more than 75 % of the hits; pixel hits
count through the seed's truth; a duplicate is any candidate whose track has another
match); the oracle's candidates on a resolution-mode event check the harness end to end.
"""
import json
import os

import numpy as np

import oracle
from lst_synth import events as E
from paper_2407_18231_gb300 import TC_DTYPE, NONE
from paper_2407_18231_gb300 import validation as V

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _tc(ot, pls=None):
    r = np.zeros(1, TC_DTYPE)
    r["ot"][0] = NONE
    r["pix"][0] = NONE
    r["ot"][0, :len(ot)] = ot
    if pls is not None:
        r["pix"][0] = [4 * pls + k for k in range(4)]
    return r


def test_match_fraction_is_the_papers():
    assert V.HIT_MATCH_FRACTION == GOLDEN["hit_match_fraction"]


def test_hand_built_candidates():
    # hits 0-4 from track 0, 5-9 from track 1, 10-11 noise
    hit_sim = np.array([0] * 5 + [1] * 5 + [-1] * 2, np.int32)
    pls_sim = np.array([1, -1], np.int32)
    tc = np.concatenate([
        _tc([0, 1, 2, 3]),           # track 0, 4/4
        _tc([5, 6, 7, 10]),          # 3/4 = 75 %: not more than 75 % -> fake
        _tc([5, 6, 7, 8, 11]),       # 4/5 = 80 % -> track 1
        _tc([1, 2, 3, 4]),           # track 0 again -> both track-0 candidates are duplicates
        _tc([10, 11], pls=0),        # 4 pixel hits of a track-1 seed + 2 noise: 4/6 -> fake
        _tc([5, 6], pls=0),          # 6/6 from track 1 -> track 1 now has two matches
        _tc([], pls=1),              # fake seed alone: fake
    ])
    m = V.match_candidates(tc, hit_sim, pls_sim)
    assert m.tolist() == [0, -1, 1, 0, -1, 1, -1]
    c = V.event_counts(tc, hit_sim, pls_sim, n_sim=3)
    assert (c["sim_selected"], c["sim_selected_matched"]) == (3, 2)
    assert (c["tc"], c["tc_fake"], c["tc_duplicate"]) == (7, 3, 4)
    r = V.rates([c, V.event_counts(tc[:1], hit_sim, pls_sim, n_sim=3, selected=np.array([1, 0, 0], bool))])
    assert r["efficiency"] == 3 / 4 and r["fake_rate"] == 3 / 8 and r["duplicate_rate"] == 4 / 8


def test_empty_inputs():
    c = V.event_counts(np.zeros(0, TC_DTYPE), np.zeros(0, np.int32), np.zeros(0, np.int32), n_sim=0)
    assert c["tc"] == 0 and c["sim_selected"] == 0
    r = V.rates([c])
    assert r["efficiency"] is None and r["fake_rate"] is None


def test_efficiency_by_bins():
    e = V.efficiency_by(np.array([0.5, 1.5, 1.6, 2.5, 9.0]), np.array([1, 1, 0, 1, 1], bool), np.array([0, 1, 2, 3]))
    assert e[0] == 1.0 and e[1] == 0.5 and e[2] == 1.0


def test_oracle_candidates_resolution_event(barrel_geom, ora_barrel):
    # prompt tracks above threshold with realistic resolution: nearly all are found, few
    # candidates are fakes or duplicates
    rng = np.random.default_rng(41)
    t = E.random_tracks(rng, 300, pt_mode="uniform", pt_lo=0.9, pt_hi=10.0, eta_max=0.8)
    ev = E.event_from_tracks(barrel_geom, t, 41, exact=False)
    r = oracle.run(ora_barrel, ev)
    tc = np.zeros(len(r["tc_type"]), TC_DTYPE)
    tc["ot"] = r["tc_ot"]
    tc["pix"] = r["tc_pix"]
    rates = V.rates([V.event_counts(tc, ev.sim, ev.pls_sim, n_sim=len(t))])
    assert rates["efficiency"] >= 0.9
    assert rates["fake_rate"] <= 0.05
    assert rates["duplicate_rate"] <= 0.1


def test_displaced_track_efficiency_ends_where_t5s_end(barrel_geom, ora_barrel):
    # Sec. 3: T5-based candidates accept displaced tracks, with an endpoint where fewer
    # than five surfaces remain.  Tracks produced inside the first layer are found; tracks
    # produced beyond the second layer (four layers left) are not.
    G = E.G  # the synthetic geometry's constants
    rng = np.random.default_rng(3)
    n = 400
    t = E.random_tracks(rng, n, pt_mode="uniform", pt_lo=2.0, pt_hi=10.0, eta_max=0.5)
    rv = rng.uniform(0, 60, n)
    ang = t["phi0"] + rng.normal(0, 0.05, n)
    t["vx"], t["vy"], t["vz"] = rv * np.cos(ang), rv * np.sin(ang), rng.normal(0, 5, n)
    ev = E.event_from_tracks(barrel_geom, t, 3, exact=False)
    r = oracle.run(ora_barrel, ev)
    tc = np.zeros(len(r["tc_type"]), TC_DTYPE)
    tc["ot"] = r["tc_ot"]
    tc["pix"] = r["tc_pix"]
    c = V.event_counts(tc, ev.sim, ev.pls_sim, n_sim=n)
    r1 = G.BARREL_R[0]
    r2 = G.BARREL_R[1] + G.BARREL_GAP[1]
    eff = V.efficiency_by(rv, c["matched_per_sim"], np.array([0.0, r1 - 1.0, r2 + 1.0, 60.0]))
    assert eff[0] >= 0.85
    assert eff[2] <= 0.05
