"""Query descriptions of the benchmark workloads (plain dicts for rel.groupby),
re-exported from the shared, arithmetic-free description module of the
inputs (synth.queries) that the oracle uses too."""
from __future__ import annotations

from synth.queries import kv_query, lineitem_query

__all__ = ["kv_query", "lineitem_query"]
