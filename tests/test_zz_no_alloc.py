"""rel_groupby_agg_static -- the group-by for callers that cannot allocate
device memory (an engine whose pool owns all GPU memory, a plugin under a
device-memory cap, a path that must not call cudaMalloc / cudaFree).  Its
hash table is a scratch array compiled into librel.so; this file checks, on
the GPU and through the C ABI, that two calls in a row give exactly what the
workspace entry point rel_groupby_agg gives (all aggregates are exact int64,
so the tolerance is zero), and that oversized requests are refused up front.

The file name makes pytest collect it last."""
import numpy as np
import pytest

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, query_to_cuda

pytestmark = pytest.mark.gpu


def _both(q_np, max_groups):
    qc = query_to_cuda(q_np)
    ref = canon_groupby(*rel.groupby(qc, flags=rel.PLAN_EXACT))
    got = canon_groupby(*rel.groupby_static(qc, max_groups=max_groups))
    return ref, got


def test_two_calls_in_a_row_match_workspace_entry_point():
    li = synth.lineitem(250_001, seed=21)
    keys, vals = synth.zipf_kv(400_003, seed=22, n_ranks=20_000)
    # call 1: few groups (thread-private tables); call 2: thousands of groups,
    # in the same shared scratch array right after call 1
    for q, max_groups in ((oracle.lineitem_query(li), 8),
                          (oracle.kv_query(keys, vals), rel.STATIC_MAX_GROUPS)):
        (rk, ra), (gk, ga) = _both(q, max_groups)
        assert len(rk) > 0
        np.testing.assert_array_equal(gk, rk)
        np.testing.assert_array_equal(ga, ra)
        ek, ea = oracle.groupby(q)
        np.testing.assert_array_equal(gk, ek)
        np.testing.assert_array_equal(ga, ea)


def test_repeated_call_sees_no_stale_state():
    keys, vals = synth.few_keys_kv(100_000, n_keys=4, seed=23)
    qc = query_to_cuda(oracle.kv_query(keys, vals))
    first = canon_groupby(*rel.groupby_static(qc, max_groups=16))
    second = canon_groupby(*rel.groupby_static(qc, max_groups=16))
    np.testing.assert_array_equal(first[0], second[0])
    np.testing.assert_array_equal(first[1], second[1])
    ek, ea = oracle.groupby(oracle.kv_query(keys, vals))
    np.testing.assert_array_equal(second[0], ek)
    np.testing.assert_array_equal(second[1], ea)


def test_sizes_beyond_the_maximum_are_rejected():
    keys, vals = synth.few_keys_kv(1000, n_keys=4, seed=24)
    qc = query_to_cuda(oracle.kv_query(keys, vals))
    for bad in (0, rel.STATIC_MAX_GROUPS + 1):
        with pytest.raises(rel.RelError) as e:
            rel.groupby_static(qc, max_groups=bad)
        assert e.value.status == rel.REL_E_UNSUPPORTED
        assert "max_groups" in str(e.value)
