"""Track-level physics metrics of a reconstruction (Sec. 3): efficiency, fake rate and
duplicate rate, with the paper's matching rule -- a simulated track matches a reconstructed
one when more than 75 % of the reconstructed track's hits come from it.

- efficiency: the fraction of the selected simulated tracks matched by at least one track
  candidate (the paper selects hard-scatter tracks; a synthetic event has no pile-up
  vertex, so the caller passes the selection, e.g. pT and |eta| bounds, as a mask);
- fake rate: the fraction of track candidates matched to no simulated track;
- duplicate rate: the fraction of track candidates matched to a simulated track that more
  than one candidate matches.

Host-side analysis of the candidates the library returns (numpy only), not part of the
reconstruction.  A candidate's hits are its outer-tracker hits (`ot`, indices into the
event's hits) and the four pixel hits of its seed (`pix` = 4 * pLS + k); a hit's truth is
`hit_sim[hit]` or `pls_sim[pLS]` (-1 for noise hits and fake seeds).
"""
from __future__ import annotations

import numpy as np

HIT_MATCH_FRACTION = 0.75  # Sec. 3
NONE = 0xFFFFFFFF


def match_candidates(tc: np.ndarray, hit_sim: np.ndarray, pls_sim: np.ndarray,
                     frac: float = HIT_MATCH_FRACTION) -> np.ndarray:
    """Per candidate the simulated track it matches (strictly more than `frac` of its hits
    from that track), or -1."""
    n = len(tc)
    if n == 0:
        return np.zeros(0, np.int64)
    ot = tc["ot"].astype(np.int64)
    pix = tc["pix"].astype(np.int64)
    hit_sim = np.asarray(hit_sim, np.int64)
    pls_sim = np.asarray(pls_sim, np.int64)
    missing = -2  # no hit in this slot (distinct from -1, a hit without a track)
    s_ot = np.where(ot != NONE, hit_sim[np.where(ot != NONE, ot, 0)] if len(hit_sim) else missing, missing)
    s_pix = np.where(pix != NONE, pls_sim[np.where(pix != NONE, pix // 4, 0)] if len(pls_sim) else missing, missing)
    m = np.concatenate([s_ot, s_pix], axis=1)
    n_hits = (m != missing).sum(1)
    counts = (m[:, :, None] == m[:, None, :]).sum(2)  # per slot: hits with the same truth
    counts = np.where(m >= 0, counts, 0)              # only real tracks can be matched
    best = counts.argmax(1)
    rows = np.arange(n)
    top = counts[rows, best]
    return np.where((n_hits > 0) & (top > frac * n_hits), m[rows, best], -1)


def event_counts(tc: np.ndarray, hit_sim: np.ndarray, pls_sim: np.ndarray, n_sim: int,
                 selected: np.ndarray | None = None, frac: float = HIT_MATCH_FRACTION) -> dict:
    """Counts behind the three rates for one event; `selected` (bool per simulated track,
    default all) is the efficiency denominator."""
    match = match_candidates(tc, hit_sim, pls_sim, frac)
    per_sim = np.bincount(match[match >= 0], minlength=n_sim) if n_sim else np.zeros(0, np.int64)
    sel = np.ones(n_sim, bool) if selected is None else np.asarray(selected, bool)
    matched = per_sim > 0
    return {
        "sim_selected": int(sel.sum()),
        "sim_selected_matched": int((sel & matched).sum()),
        "tc": int(len(tc)),
        "tc_fake": int((match < 0).sum()),
        "tc_duplicate": int(((match >= 0) & (per_sim[np.maximum(match, 0)] > 1)).sum()) if n_sim else 0,
        "matched_per_sim": matched,
    }


def rates(counts: list[dict]) -> dict:
    """Efficiency, fake and duplicate rate over several events' counts."""
    s = {k: sum(c[k] for c in counts) for k in ("sim_selected", "sim_selected_matched", "tc", "tc_fake",
                                                 "tc_duplicate")}
    return {
        "efficiency": s["sim_selected_matched"] / s["sim_selected"] if s["sim_selected"] else None,
        "fake_rate": s["tc_fake"] / s["tc"] if s["tc"] else None,
        "duplicate_rate": s["tc_duplicate"] / s["tc"] if s["tc"] else None,
        **s,
    }


def efficiency_by(values: np.ndarray, matched: np.ndarray, bins: np.ndarray) -> np.ndarray:
    """Efficiency per bin of `values` (e.g. simulated pT or production radius): matched /
    selected tracks in each bin, NaN for an empty bin."""
    values = np.asarray(values, np.float64)
    idx = np.digitize(values, bins) - 1
    ok = (idx >= 0) & (idx < len(bins) - 1)
    den = np.bincount(idx[ok], minlength=len(bins) - 1).astype(np.float64)
    num = np.bincount(idx[ok], weights=np.asarray(matched, np.float64)[ok], minlength=len(bins) - 1)
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / den
