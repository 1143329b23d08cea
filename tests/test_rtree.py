"""The CPU R-tree baseline (the paper's CPU comparator, Sec. 5: r consecutive segments of a
trajectory per 4-D box, an R-tree over the boxes, OpenMP queries) returns the oracle's match set
exactly: on the tiny configuration in full at several distances, and on random sets whose
queries are not database segments, with a partial query interval."""
import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import workloads
from tests.cases import random_segments


def _same(a, b):
    for k in ("q_idx", "e_idx", "t_in", "t_out"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_rtree_equals_the_oracle_on_the_tiny_configuration(r):
    w = workloads.tiny()
    tree = oracle.RTree(w.db, r)
    groups, levels = tree.shape()
    # 1,000 trajectories of 20 segments: ceil(20 / r) groups each, never across trajectories
    assert groups == 1000 * -(-20 // r) and levels >= 2
    for d in (1.0, 5.0, 12.0):
        ref = oracle.search(w.db, w.queries, w.t_start, w.t_end, d)
        got = tree.search(w.queries, w.t_start, w.t_end, d)
        _same(got, ref)
        hits, tests, qsegs = tree.count(w.queries, w.t_start, w.t_end, d, threads=4)
        assert hits == ref["q_idx"].size
        assert 0 < tests < ref["n_tests"]  # the tree prunes in space as well as in time
        assert qsegs == int(np.sum(np.minimum(w.queries.t1, w.t_end) >
                                   np.maximum(w.queries.t0, w.t_start)))


def test_rtree_equals_the_oracle_on_random_sets():
    rng = np.random.default_rng(17)
    db = random_segments(rng, 3000, box=30.0, stationary_frac=0.1)
    q = random_segments(rng, 300, box=30.0, stationary_frac=0.1)
    tree = oracle.RTree(db, 1)
    for d, ts, te in ((0.5, -1e9, 1e9), (2.0, 3.0, 7.5), (4.0, 0.0, 12.0)):
        _same(tree.search(q, ts, te, d), oracle.search(db, q, ts, te, d))
    tree.free()
