"""Query descriptions of the benchmark workloads: which columns are keys,
filters and aggregate inputs (plain dicts; no arithmetic of the method).
Shared by the oracle, the GPU binding's workload helpers and the bench, so
the two sides cannot drift apart.

lineitem_query: the fused filter + group-by the paper profiles as its
aggregation example (Sec. 7): keep date <= date_hi, group by (flag, status),
sum(qty), sum(price), sum(price * (100 - disc)),
sum(price * (100 - disc) * (100 + tax)), count.
kv_query: aggregates of one int64 value column grouped by one key column.
Columns may be numpy arrays or CUDA tensors.
"""
from __future__ import annotations


def lineitem_query(li: dict, date_hi: int = 2430) -> dict:
    cols = [li["flag"], li["status"], li["qty"], li["price"], li["disc"], li["tax"], li["date"]]
    return {"cols": cols, "keys": [0, 1], "preds": [(6, -(2**31), date_hi)],
            "aggs": [("sum", 2, []), ("sum", 3, []), ("sum", 3, [(4, 100, -1)]),
                     ("sum", 3, [(4, 100, -1), (5, 100, 1)]), ("count", 2, [])]}


def kv_query(keys, vals, ops=("sum", "count", "min", "max")) -> dict:
    return {"cols": [keys, vals], "keys": [0], "preds": [], "aggs": [(o, 1, []) for o in ops]}
