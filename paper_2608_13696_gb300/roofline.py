"""Instruction roofline (Sec. 2.2) and the utilisation figures reported per kernel.

The paper plots warp instructions per second against instruction intensity,
warp instructions per 32-byte DRAM sector.  The flat roof is the warp
instruction throughput  N_SM x N_SMSP x measured SM clock  (one issue per
sub-partition per cycle); the slanted roof is DRAM bandwidth in sectors per
second.  A kernel left of the ridge is memory bound, right of it compute
bound, and a bottleneck counts as saturated at >= 75 % use (Sec. 5, Table 6).
"""
from __future__ import annotations

SECTOR_BYTES = 32
SATURATED = 0.75


def inst_throughput(n_sm: int, smsp_per_sm: int, clock_hz: float) -> float:
    """Warp instructions per second with every SM issuing (Sec. 2.2)."""
    return float(n_sm) * float(smsp_per_sm) * float(clock_hz)


def ridge(inst_per_s: float, dram_bytes_per_s: float) -> float:
    """Instruction intensity (warp inst per sector) where the two roofs meet."""
    return inst_per_s / (dram_bytes_per_s / SECTOR_BYTES)


def intensity(warp_inst: float, dram_bytes: float) -> float:
    """Warp instructions per DRAM sector moved."""
    return float("inf") if dram_bytes <= 0 else warp_inst / (dram_bytes / SECTOR_BYTES)


def bound(inst_per_sector: float, ridge_inst_per_sector: float) -> str:
    return "memory" if inst_per_sector < ridge_inst_per_sector else "compute"


def attainable(inst_per_sector: float, inst_per_s: float, dram_bytes_per_s: float) -> float:
    """Roof height (warp inst/s) at a given instruction intensity."""
    return min(inst_per_s, inst_per_sector * dram_bytes_per_s / SECTOR_BYTES)


def full_wave(n_ctas: int, ctas_per_sm: int, n_sm: int) -> bool:
    """Whether a launch fills every SM at least once (Sec. 6.1)."""
    return n_ctas >= ctas_per_sm * n_sm


def report(*, seconds: float, algo_bytes: float, peak_bytes_per_s: float,
           warp_inst: float | None = None, n_sm: int | None = None,
           clock_hz: float | None = None, dram_bytes: float | None = None,
           rows: float | None = None) -> dict:
    """Fractions of the HBM roof (algorithmic bytes / time / peak) and, when the
    issued warp instructions are known, of the instruction-issue roof."""
    out = {"seconds": seconds, "gbps": algo_bytes / seconds / 1e9,
           "hbm_frac": algo_bytes / seconds / peak_bytes_per_s}
    if rows:
        out["rows_per_s"] = rows / seconds
    if warp_inst is not None and n_sm and clock_hz:
        roof = inst_throughput(n_sm, 4, clock_hz)
        out["issue_frac"] = warp_inst / seconds / roof
        out["inst_per_byte"] = warp_inst / algo_bytes if algo_bytes else None
        if rows:
            out["warp_inst_per_row"] = warp_inst / rows
        if dram_bytes:
            out["inst_per_sector"] = intensity(warp_inst, dram_bytes)
            out["ridge"] = ridge(roof, peak_bytes_per_s)
            out["bound"] = bound(out["inst_per_sector"], out["ridge"])
    return out
