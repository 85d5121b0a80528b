"""GPU parity of the learned T5 selection.

With the shipped network (lst_set_t5_selection) every object list of the CUDA chain equals
the oracle's chain with the same weights, element by element and bit for bit -- the
network is binary32 with one fixed summation order on both sides, so the tolerance is
zero.  Switching the selection on and off takes effect on the next run (graphs are
captured again); the serving loop and the batch slots follow it too; bad weights are
refused and leave the context as it was.
"""
import numpy as np
import pytest

import lst_synth as S
import oracle
import paper_2407_18231_gb300 as lst
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weights():
    lst.build()
    return lst.load_t5_mlp()


@pytest.fixture(scope="module")
def ora_net(full_geom, weights):
    og = oracle.Geometry(full_geom.modules)
    oracle.set_t5_mlp(og, weights)
    return og


@pytest.fixture(scope="module")
def sess_net(full_geom, weights):
    s = lst.Session(full_geom.modules, keep_objects=True)
    s.set_t5_selection(weights)
    yield s
    s.close()


@pytest.mark.parametrize("n_tracks", [1000, 4000])
def test_learned_t5_pu200_parity(sess_net, ora_net, n_tracks):
    ev = S.make_event("pu200", 30, n_tracks=n_tracks, with_pls=True)
    compare(sess_net, sess_net.run_event(ev), oracle.run(ora_net, ev), ev, f"learned pu200 {n_tracks}")


def test_learned_t5_highocc_full_size_parity(sess_net, ora_net):
    ev = S.make_event("highocc", 2)
    ora = oracle.run(ora_net, ev)
    compare(sess_net, sess_net.run_event(ev), ora, ev, "learned highocc")
    assert len(ora["t5"]) > 1000


def test_learned_t5_tilted_parity(tilted_geom, weights):
    og = oracle.Geometry(tilted_geom.modules)
    oracle.set_t5_mlp(og, weights)
    s = lst.Session(tilted_geom.modules, keep_objects=True)
    s.set_t5_selection(weights)
    evs = [S.make_event("pu200", 35, with_pls=True, realistic=True),
           S.make_event("highocc", 4, n_tracks=5000, realistic=True)]
    for i, (ev, rid) in enumerate(zip(evs, s.run_batch(evs))):
        compare(s, rid, oracle.run(og, ev), ev, f"learned tilted {i}")
    s.close()


def test_switching_the_selection_recaptures(full_geom, ora_full, ora_net, weights):
    """Cuts, network, cuts again on one context and one batch (the graph path): each run
    equals the oracle with the selection then in force, and the two selections differ."""
    s = lst.Session(full_geom.modules, keep_objects=True)
    evs = [S.make_event("pu200", 31 + i, n_tracks=1500, with_pls=True) for i in range(3)]
    evs.append(S.make_event("highocc", 3, n_tracks=4000))
    n_t5 = {}
    for phase, (w, og) in enumerate(((None, ora_full), (weights, ora_net), (None, ora_full))):
        s.set_t5_selection(w)
        ids = s.run_batch(evs)
        n_t5[phase] = 0
        for i, (ev, rid) in enumerate(zip(evs, ids)):
            compare(s, rid, oracle.run(og, ev), ev, f"phase {phase} event {i}")
            n_t5[phase] += len(s.objects(rid, lst.OBJ_T5))
            s.release(rid)
    assert n_t5[0] == n_t5[2] > n_t5[1] > 0
    s.close()


def test_learned_t5_serving_and_async_slots(full_geom, ora_net, weights):
    """The serving loop's slots and the two submit/collect slots run the selection too."""
    s = lst.Session(full_geom.modules)
    s.set_t5_selection(weights)
    evs = [S.make_event("pu200", 40 + i, n_tracks=1200, with_pls=True) for i in range(6)]
    refs = [oracle.run(ora_net, ev) for ev in evs]
    arrival = np.linspace(0.0, 0.01, len(evs))
    _, _, ids, _ = s.serve_replay(evs, arrival, n_slots=2, max_batch=2, keep_results=True)
    for ev, ref, rid in zip(evs, refs, ids):
        tc = s.candidates(rid)
        assert np.array_equal(tc["ot"], ref["tc_ot"]) and tc["score"].tobytes() == ref["tc_score"].tobytes()
    t = s.submit_batch(evs[:3])
    ids = s.collect_batch(t)
    for ref, rid in zip(refs, ids):
        tc = s.candidates(rid)
        assert np.array_equal(tc["type"], ref["tc_type"]) and np.array_equal(tc["ot"], ref["tc_ot"])
    s.close()


def test_bad_weights_refused(full_geom, ora_full, weights):
    s = lst.Session(full_geom.modules, keep_objects=True)
    with pytest.raises(lst.LstError) as e:
        s.set_t5_selection(weights[:-1])
    assert e.value.status == -1 and "433" in str(e.value)
    w = weights.copy()
    w[3] = np.inf
    with pytest.raises(lst.LstError) as e:
        s.set_t5_selection(w)
    assert e.value.status == -1 and "not finite" in str(e.value)
    ev = S.make_event("pu200", 45, n_tracks=600, with_pls=True)  # still the cuts
    compare(s, s.run_event(ev), oracle.run(ora_full, ev), ev, "after refused weights")
    s.close()
