"""Shared helpers of the GPU parity tests: move seeded numpy inputs to the GPU
and put results in canonical order (group-by: ascending key; join: ascending
(probe_idx, build_idx)) so they compare element by element with the oracle."""
import numpy as np
import torch


def cuda(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def query_to_cuda(q: dict) -> dict:
    out = dict(q)
    out["cols"] = [cuda(c) for c in q["cols"]]
    return out


def canon_groupby(keys: torch.Tensor, aggs):
    k = keys.cpu().numpy()
    order = np.argsort(k, kind="stable")
    a = np.stack([x.cpu().numpy()[order] for x in aggs]) if aggs else np.zeros((0, len(k)), np.int64)
    return k[order], a


def canon_join(pi, bi, pay):
    pi, bi, pay = pi.cpu().numpy(), bi.cpu().numpy(), pay.cpu().numpy()
    order = np.lexsort((bi, pi))
    return pi[order], bi[order], pay[order]
