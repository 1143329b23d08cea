"""The device-side timeout path of the pair kernel. Every wait of the kernel on a bulk copy is
bounded by the GPU's global timer; when one runs out, the kernel records a timeout in the search's
status word, waits (bounded) for its own copies in flight and returns. Here a test hook makes one
warp of the next plain search's count pass wait 1 ms on a barrier phase that nothing completes
(no copy is involved, nothing faults): the search must end with TS_ERR_TIMEOUT, and the next
search on the same index must return the oracle's rows."""
import time

import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads

from tests import parity

pytestmark = pytest.mark.gpu

TS_ERR_TIMEOUT = 5


@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal"])
def test_bounded_wait_times_out_and_the_context_stays_usable(kind):
    w = workloads.tiny()
    db = w.db
    q = w.queries.take(np.arange(400))
    idx = api.ts_build_index(db, kind=kind)
    ref = oracle.search(db, q, w.t_start, w.t_end, 5.0)
    api.ts_debug_inject_stall(1_000_000)  # 1 ms
    t0 = time.perf_counter()
    with pytest.raises(api.TsError) as e:
        api.ts_search(idx, q, 5.0, w.t_start, w.t_end)
    assert e.value.status == TS_ERR_TIMEOUT, str(e.value)
    assert "wait" in str(e.value)
    assert time.perf_counter() - t0 < 30.0
    # the hook is used up: the next searches on the same index are whole and correct
    for _ in range(2):
        got = api.ts_search(idx, q, 5.0, w.t_start, w.t_end).to_host(sort=True)
        parity.compare(got, ref, db, q, w.t_start, w.t_end, 5.0)
    idx.free()


def test_stall_hook_rejects_unbounded_limits():
    with pytest.raises(api.TsError) as e:
        api.ts_debug_inject_stall(0)
    assert e.value.status == 1
    with pytest.raises(api.TsError) as e:
        api.ts_debug_inject_stall(2_000_000_000)
    assert e.value.status == 1
