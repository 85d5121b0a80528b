"""Pins of the learned T5 selection in the oracle.

The network's inputs are checked against float64 values computed here from the anchors'
coordinates and against the cut conditions they are built from (an input x / (x + y) is
above 1/2 exactly when x > y); the network against its matrix definition in float64; the
chain with a network against the chain with the cuts through weights that reproduce the
cuts; and the shipped weights against the held-out record their training script wrote.
"""
import json

import numpy as np
import pytest

import lst_synth as S
import oracle
from helix_cases import RMIN, clean_track, curvature, outward, points, shift_doublet, edited

NF, NH = oracle.T5_NF, oracle.T5_NH
ALL_T5 = 15
KMAX = 1.0 / (0.95 * RMIN)


def unpack(w):
    w = np.asarray(w, np.float64)
    o = 0
    W1 = w[o:o + NH * NF].reshape(NH, NF); o += NH * NF
    b1 = w[o:o + NH]; o += NH
    W2 = w[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = w[o:o + NH]; o += NH
    w3 = w[o:o + NH]; o += NH
    return W1, b1, W2, b2, w3, w[o]


def net64(w, f):
    """The network's definition in float64, and the same network on absolute values (a
    bound on every partial sum, for the rounding tolerance)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    f = np.asarray(f, np.float64)
    h2 = np.maximum(W2 @ np.maximum(W1 @ f + b1, 0) + b2, 0)
    mag = abs(b3) + np.abs(w3) @ (np.abs(b2) + np.abs(W2) @ (np.abs(b1) + np.abs(W1) @ np.abs(f)))
    return w3 @ h2 + b3, mag


def cut_network():
    """Weights with z = 1/2 - f0 - relu(f1 - f0) = 1/2 - max(f0, f1): z > 0 exactly when
    d1 < rhs1 and d2 < rhs2, the two curvature-agreement cuts (up to ties)."""
    W1, b1 = np.zeros((NH, NF)), np.zeros(NH)
    W2, b2 = np.zeros((NH, NH)), np.zeros(NH)
    w3 = np.zeros(NH)
    W1[0, 0] = 1.0
    W1[1, 0], W1[1, 1] = -1.0, 1.0
    W2[0, 0] = W2[1, 1] = 1.0
    w3[0] = w3[1] = -1.0
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [0.5]]).astype(np.float32)


@pytest.fixture(scope="module")
def og_net(full_geom):
    """An oracle geometry of its own (the model is geometry state)."""
    return oracle.Geometry(full_geom.modules)


def _candidates(r, ev):
    """Every T3 pair sharing an MD: (module ids, anchor points, MD indices)."""
    md, t3 = r["md"], r["t3"]
    P = np.stack([ev.x, ev.y, ev.z], 1)
    starting = {}
    for k, t in enumerate(t3):
        starting.setdefault(int(t[0]), []).append(k)
    for t in t3:
        for k2 in starting.get(int(t[2]), []):
            ch = [int(t[0]), int(t[1]), int(t[2]), int(t3[k2][1]), int(t3[k2][2])]
            yield md[ch, 0], P[md[ch, 1]], ch


# ---------------------------------------------------------------- the network
def test_network_matches_its_matrix_definition():
    """Random weights and inputs: the binary32 network equals relu/affine algebra in float64
    within the rounding of its partial sums; with every hidden unit switched off (negative
    first-layer biases on non-negative inputs, zero weights) z is b3 exactly."""
    rng = np.random.default_rng(5)
    for _ in range(400):
        w = rng.normal(0, 1, oracle.T5_NPARAM).astype(np.float32)
        f = rng.random(NF).astype(np.float32)
        z = oracle.t5_logit(w, f)
        z64, mag = net64(w, f)
        assert abs(float(z) - z64) <= 1e-5 * mag + 1e-30, (z, z64, mag)
    w = np.zeros(oracle.T5_NPARAM, np.float32)
    w[NH * NF:NH * NF + NH] = -1.0
    w[-1] = np.float32(-0.3125)
    assert oracle.t5_logit(w, rng.random(NF)) == np.float32(-0.3125)


def test_network_layout_single_paths():
    """One path f_i -> h1_j -> h2_k -> z with unit weights carries f_i alone: pins which index
    of each weight matrix is the unit and which the input."""
    rng = np.random.default_rng(6)
    for _ in range(40):
        i, j, k = int(rng.integers(NF)), int(rng.integers(NH)), int(rng.integers(NH))
        W1, b1 = np.zeros((NH, NF)), np.zeros(NH)
        W2, b2, w3 = np.zeros((NH, NH)), np.zeros(NH), np.zeros(NH)
        W1[j, i] = 1.0
        W2[k, j] = 2.0
        w3[k] = 3.0
        w = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [0.0]]).astype(np.float32)
        f = np.zeros(NF, np.float32)
        f[i] = 0.25
        assert oracle.t5_logit(w, f) == np.float32(1.5)
        f[i] = 0.0
        f[(i + 1) % NF] = 0.25
        assert oracle.t5_logit(w, f) == np.float32(0.0)


def test_bad_weights_rejected(og_net):
    with pytest.raises(ValueError):
        oracle.set_t5_mlp(og_net, np.zeros(oracle.T5_NPARAM - 1, np.float32))
    w = np.zeros(oracle.T5_NPARAM, np.float32)
    w[7] = np.nan
    with pytest.raises(ValueError):
        oracle.set_t5_mlp(og_net, w)
    oracle.set_t5_mlp(og_net, None)


# ---------------------------------------------------------------- the inputs
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_curvature_inputs_against_float64(seed, barrel_geom, ora_barrel):
    """Five anchors of a clean 2-8 GeV barrel track, each doublet moved outward by up to 0.05
    cm: f0..f5 from float64 curvatures of the anchors (the triple curvature of Menger,
    2 cross / product of the sides), flat-barrel point errors 8 x 0.01 cm / span^2, the cut
    tolerance 5 % of the curvature sum + errors + 1e-4 / cm, and k_max = 1 / (0.95 Rmin)."""
    rng = np.random.default_rng(seed)
    n = 0
    for trial in range(12):
        while True:  # some pseudorapidities put a layer's crossing on a z-bin edge
            pt, eta = float(rng.uniform(2.0, 8.0)), float(rng.uniform(-0.4, 0.4))
            try:
                t, ev, d = clean_track(barrel_geom, pt, eta, 6, phis=np.linspace(0.11, 6.1, 13) + rng.uniform(0, 0.4))
                break
            except AssertionError:
                continue
        ch = {}
        for x in d[:5]:
            p = points(ev)[x[1]]
            ch.update(shift_doublet(ev, x, dxy=float(rng.uniform(-0.05, 0.05)) * outward(t, p)))
        e2 = edited(ev, ch)
        P = points(e2)
        A = [P[x[1]] for x in d[:5]]
        f = oracle.t5_features(ora_barrel, [x[0] for x in d[:5]], np.array(A, np.float32))
        kin, kout = curvature(A[0], A[1], A[2]), curvature(A[2], A[3], A[4])
        kbr, kfu = curvature(A[1], A[2], A[3]), curvature(A[0], A[2], A[4])

        def err(p, s):
            return 0.08 / ((p[0] - s[0]) ** 2 + (p[1] - s[1]) ** 2)

        tin, tout, tbr, tfu = err(A[0], A[2]), err(A[2], A[4]), err(A[1], A[3]), err(A[0], A[4])
        d1, d2 = abs(kin - kout), abs(kbr - kfu)
        rhs1 = 0.05 * (abs(kin) + abs(kout)) + tin + tout + 1e-4
        rhs2 = 0.05 * (abs(kbr) + abs(kfu)) + tbr + tfu + 1e-4
        want = [d1 / (d1 + rhs1), d2 / (d2 + rhs2), d1 / (d1 + abs(kin) + abs(kout) + 1e-4),
                d2 / (d2 + abs(kbr) + abs(kfu) + 1e-4),
                (tin + tout) / (tin + tout + abs(kin) + abs(kout) + 1e-4), abs(kfu) / KMAX]
        assert np.allclose(f[:6], want, rtol=0, atol=2e-3), (trial, f[:6], want)
        n += 1
    assert n == 12


@pytest.mark.parametrize("realistic", [False, True])
def test_ratio_inputs_match_the_conditions_they_come_from(realistic, full_geom, ora_full, tilted_geom, ora_tilted):
    """Over every T3 pair of a PU200-like event: f0 > 1/2 exactly when the inner/outer
    condition fails, f1 > 1/2 when bridge/full fails, f6 > 1/2 when (a, c, e) is not straight
    in r-z, f7 > 1/2 when (b, c, d) is not (the T3 r-z condition on b, c, d).  Inputs within
    1e-6 of 1/2 are rounding ties and skipped."""
    og = ora_tilted if realistic else ora_full
    ev = S.make_event("pu200", 11, n_tracks=1500, realistic=realistic)
    r = oracle.run(og, ev)
    P = np.stack([ev.x, ev.y, ev.z], 1)
    md = r["md"]
    fails = np.zeros(4, np.int64)
    n = 0
    for mods, pts, ch in _candidates(r, ev):
        f = oracle.t5_features(og, mods, pts)
        mask, _, _ = oracle.t5_eval(og, mods, pts)
        c, cu = ch[2], md[ch[2], 2]
        rz_bcd = oracle.t3_eval(og, (mods[1], mods[2], mods[3]), pts[1], pts[2], P[cu], pts[3]) & oracle.T3_RZ
        for k, (x, ok) in enumerate(((f[0], mask & oracle.T5_INOUT), (f[1], mask & oracle.T5_BRFULL),
                                     (f[6], mask & oracle.T5_RZ), (f[7], rz_bcd))):
            if abs(float(x) - 0.5) < 1e-6:
                continue
            assert (x > 0.5) == (not ok), (ch, k, x, mask)
            fails[k] += x > 0.5
        assert np.all((f >= 0) & ((f < 1) | (np.arange(NF) == 5)))  # f5 = |k_full| / k_max is unbounded
        n += 1
    assert n > 2000 and np.all(fails > 20), (n, fails)


# ---------------------------------------------------------------- the chain with a network
@pytest.mark.parametrize("realistic", [False, True])
def test_network_reproducing_the_cuts_gives_the_cut_chain(realistic, full_geom, tilted_geom):
    """With weights computing z = 1/2 - max(f0, f1), the chain's T5s (scores, curvatures),
    pT5s, duplicate removal and track candidates equal the cut chain's, and every candidate's
    decision bits do: bits 0 and 1 both carry the network's decision, bits 2 and 3 (radius,
    r-z) stay."""
    geom = tilted_geom if realistic else full_geom
    og = oracle.Geometry(geom.modules)
    ev = S.make_event("pu200", 12, n_tracks=2500, with_pls=True, realistic=realistic)
    cut = oracle.run(og, ev)
    oracle.set_t5_mlp(og, cut_network())
    net = oracle.run(og, ev)
    for k in ("t5", "t5_score", "t5_kfull", "pt5", "pt5_score", "alive_t5", "alive_pt5", "tc_type", "tc_obj",
              "tc_ot", "tc_pix"):
        assert np.array_equal(cut[k], net[k]), k
    assert len(cut["t5"]) > 500
    n_diff = 0
    for mods, pts, ch in _candidates(cut, ev):
        m_net, _, _ = oracle.t5_eval(og, mods, pts)
        oracle.set_t5_mlp(og, None)
        m_cut, _, _ = oracle.t5_eval(og, mods, pts)
        oracle.set_t5_mlp(og, cut_network())
        assert (m_net & 1) == ((m_net >> 1) & 1)
        assert (m_net & 12) == (m_cut & 12)
        assert ((m_net & 3) == 3) == ((m_cut & 3) == 3)
        n_diff += (m_cut & 3) not in (0, 3)
    assert n_diff > 100  # candidates failing exactly one of the two cuts were seen


def test_network_decision_is_z_positive(full_geom):
    """A constant network: b3 = +1 accepts every candidate passing radius and r-z, b3 = -1
    (and b3 = 0: z > 0 is strict) none."""
    og = oracle.Geometry(full_geom.modules)
    ev = S.make_event("pu200", 13, n_tracks=800)
    r0 = oracle.run(og, ev)
    w = np.zeros(oracle.T5_NPARAM, np.float32)
    counts = {}
    for b3 in (1.0, 0.0, -1.0):
        w[-1] = b3
        oracle.set_t5_mlp(og, w)
        counts[b3] = len(oracle.run(og, ev)["t5"])
    oracle.set_t5_mlp(og, None)
    hard = 0
    for mods, pts, _ in _candidates(r0, ev):
        m, _, _ = oracle.t5_eval(og, mods, pts)
        hard += (m & 12) == 12
    assert counts[1.0] == hard > len(r0["t5"]) and counts[0.0] == counts[-1.0] == 0


# ---------------------------------------------------------------- the shipped weights
def _shipped():
    import paper_2407_18231_gb300 as lst
    with open(lst.T5_MLP_PATH) as f:
        return json.load(f), lst.load_t5_mlp()


def test_shipped_weights_well_formed():
    rec, w = _shipped()
    assert w.dtype == np.float32 and w.size == oracle.T5_NPARAM and np.all(np.isfinite(w))
    assert rec["hidden"] == NH and len(rec["inputs"]) == NF and rec["decision"] == "z > 0"


def test_shipped_weights_reproduce_their_heldout_record(full_geom):
    """The held-out figures stored beside the weights come back exactly from the oracle on
    those events, and they show what the network is for: at least 99.5 % of the true T5
    candidates kept and at most a third of the cuts' other candidates accepted."""
    from oracle import train_t5_mlp as T
    rec, w = _shipped()
    h = rec["heldout"]
    og = oracle.Geometry(full_geom.modules)
    X, Y, CUT = T.collect(og, range(*h["events"]))
    z = T.logits(w, X)
    assert len(Y) == h["candidates"] and int(Y.sum()) == h["true"]
    assert float(np.mean(z[Y] > 0)) == h["true_kept"]
    assert int(np.sum((z > 0) & ~Y)) == h["other_accepted"]
    assert int(np.sum(CUT & ~Y)) == h["cut_other_accepted"]
    assert h["true_kept"] >= 0.995 and h["other_accepted"] * 3 <= h["cut_other_accepted"]
    # the chain with the network accepts exactly the candidates with z > 0 among those
    # passing radius and r-z (one event)
    ev = S.make_event("pu200", h["events"][0])
    oracle.set_t5_mlp(og, w)
    r = oracle.run(og, ev)
    n_acc = 0
    for mods, pts, _ in _candidates(r, ev):
        m, _, _ = oracle.t5_eval(og, mods, pts)
        f = oracle.t5_features(og, mods, pts)
        if (m & 12) == 12:
            assert ((m & 3) == 3) == (oracle.t5_logit(w, f) > 0)
        n_acc += m == ALL_T5
    assert n_acc == len(r["t5"])
