"""Comparison of a GPU result with the oracle under the acceptance rule of the search:

* the (query, entry) pair set equals the oracle's, except pairs whose minimum separation lies
  within 1e-9 * d of d (near-tangent pairs, where both FP64 evaluations may round either way);
* for every common pair |t_in - t_in_oracle| and |t_out - t_out_oracle| are at most 1e-9 times
  the pair's overlap duration;
* no pair is reported twice.
"""
from __future__ import annotations

import numpy as np

import oracle

REL_D = 1e-9
REL_T = 1e-9


def _keys(q, e):
    return q.astype(np.uint64) << np.uint64(32) | e.astype(np.uint64)


def overlap_duration(db, queries, qi, ei, Ts, Te):
    lo = np.maximum(np.maximum(queries.t0[qi], db.t0[ei]), Ts)
    hi = np.minimum(np.minimum(queries.t1[qi], db.t1[ei]), Te)
    return hi - lo


def compare(got: dict, ref: dict, db, queries, Ts, Te, d, allow_exempt=True):
    """Assert parity; returns a dict of diagnostics (worst errors, exempt pairs)."""
    kg = _keys(got["q_idx"], got["e_idx"])
    kr = _keys(ref["q_idx"], ref["e_idx"])
    if np.array_equal(kg, kr) and (kg.size < 2 or bool(np.all(kg[1:] > kg[:-1]))):
        # the same strictly increasing keys (both sides sorted): no duplicates, no differences
        T = overlap_duration(db, queries, got["q_idx"].astype(np.int64),
                             got["e_idx"].astype(np.int64), Ts, Te)
        e_in = np.abs(got["t_in"] - ref["t_in"])
        e_out = np.abs(got["t_out"] - ref["t_out"])
        worst_in = float((e_in / T).max()) if T.size else 0.0
        worst_out = float((e_out / T).max()) if T.size else 0.0
        assert np.all(e_in <= REL_T * T), f"t_in error {worst_in:.3e} of the overlap"
        assert np.all(e_out <= REL_T * T), f"t_out error {worst_out:.3e} of the overlap"
        assert np.all(got["t_in"] <= got["t_out"])
        return {"rows": int(kg.size), "exempt": 0, "worst_in": worst_in, "worst_out": worst_out,
                "bit_exact": bool(np.array_equal(got["t_in"], ref["t_in"])
                                  and np.array_equal(got["t_out"], ref["t_out"]))}
    assert np.unique(kg).size == kg.size, "duplicate (query, entry) rows"
    only_g = np.setdiff1d(kg, kr)
    only_r = np.setdiff1d(kr, kg)
    exempt = 0
    for keys in (only_g, only_r):
        if keys.size == 0:
            continue
        qi = (keys >> np.uint64(32)).astype(np.int64)
        ei = (keys & np.uint64(0xffffffff)).astype(np.int64)
        _, _, _, smin = oracle.eval_pairs(db, queries, qi, ei, Ts, Te, d)
        bad = np.abs(smin - d) > REL_D * d
        assert allow_exempt and not bad.any(), (
            f"{int(bad.sum())} pairs differ outside the near-tangent band: "
            f"{list(zip(qi[bad][:5], ei[bad][:5], smin[bad][:5]))}")
        exempt += keys.size
    common, ig, ir = np.intersect1d(kg, kr, return_indices=True)
    qi = (common >> np.uint64(32)).astype(np.int64)
    ei = (common & np.uint64(0xffffffff)).astype(np.int64)
    T = overlap_duration(db, queries, qi, ei, Ts, Te)
    e_in = np.abs(got["t_in"][ig] - ref["t_in"][ir])
    e_out = np.abs(got["t_out"][ig] - ref["t_out"][ir])
    worst_in = float((e_in / T).max()) if T.size else 0.0
    worst_out = float((e_out / T).max()) if T.size else 0.0
    assert np.all(e_in <= REL_T * T), f"t_in error {worst_in:.3e} of the overlap"
    assert np.all(e_out <= REL_T * T), f"t_out error {worst_out:.3e} of the overlap"
    assert np.all(got["t_in"] <= got["t_out"])
    return {"rows": int(kg.size), "exempt": int(exempt), "worst_in": worst_in,
            "worst_out": worst_out,
            "bit_exact": bool(np.array_equal(got["t_in"][ig], ref["t_in"][ir])
                              and np.array_equal(got["t_out"][ig], ref["t_out"][ir]))}
