"""Autotuner: every candidate it times returns the same rows, the choice is cached per workload
and GPU, and a plan built with the chosen parameters returns the plain search's rows."""
import json

import numpy as np
import pytest

from paper_1410_2698_gb300 import api, autotune, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal", "spatial"])
def test_autotune_choice_and_cache(kind, tmp_path):
    w = workloads.tiny()
    reqs = [(w.queries, d, w.t_start, w.t_end) for d in (1.0, 5.0)]
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(w.db, reqs, kind, cache_path=cache, repeats=1, max_rows=1 << 22,
                         index_budget=3)
    assert best["tile_records"] in autotune.TILES
    assert best["trials"] and all(t["s"] > 0 for t in best["trials"])
    with open(cache) as f:
        stored = json.load(f)
    assert len(stored) == 1
    again = autotune.tune(w.db, reqs, kind, cache_path=cache)  # served from the cache
    assert again == json.loads(json.dumps(best))
    # the tuned configuration returns the plain rows
    idx = api.ts_build_index(w.db, kind=kind, **best["index"])
    plan = api.BatchPlan(idx, max_requests=len(reqs), max_queries=2 * w.queries.n,
                         max_rows=1 << 22, tile_records=best["tile_records"],
                         pair_blocks=best["pair_blocks"])
    plan.run(reqs)
    st = plan.wait()
    assert not st["overflow"] and st["rows"] == best["rows"]
    for r, (q, d, ts, te) in enumerate(reqs):
        got = plan.request_to_host(r, sort=True)
        ref = api.ts_search(idx, q, d, ts, te).to_host(sort=True)
        for k in ("q_idx", "e_idx", "t_in", "t_out"):
            assert np.array_equal(got[k], ref[k]), k
    plan.free()
    idx.free()
