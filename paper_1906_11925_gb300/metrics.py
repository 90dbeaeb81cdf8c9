"""Throughput and roofline arithmetic used by the benchmark.

Site updates per second (SUPS) is the paper's metric (Section 4, Table III):
the number of fluid sites times the number of time steps, divided by the
wall time.  Bytes per site update are the algorithmic traffic of one pull
step on the sparse site list (see ``bytes_per_site_update``).
"""
from __future__ import annotations


def sups(n_sites: int, steps: int, seconds: float) -> float:
    """Site updates per second: n_sites * steps / seconds."""
    return float(n_sites) * float(steps) / float(seconds)


def msups(n_sites: int, steps: int, seconds: float) -> float:
    return sups(n_sites, steps, seconds) / 1e6


def bytes_per_site_update(q: int, storage: str, streaming: str = "pull") -> int:
    """Algorithmic HBM bytes of one fused collide-and-stream update:
    q populations read and q written (4 B each in fp32, 2 B in the 16-bit
    deviation forms, fp16 or int16) plus the int32 neighbour entries (q - 1;
    the rest population needs none).  Pull streaming reads the table every
    step; the AA pattern only on odd steps, so its average over a step pair
    is (q - 1) * 2 B.  The fused AA step pair ("aa_pairs", slab chunks) reads
    and writes the populations once per pair, the odd step finding the even
    step's output in L2: per step half of 2 q elem + 4 (q - 1)."""
    elem = {"fp32": 4, "fp16": 2, "i16": 2}[storage]
    if streaming == "aa_pairs":
        return (2 * q * elem + 4 * (q - 1)) // 2
    table = {"pull": 4 * (q - 1), "aa": 2 * (q - 1)}[streaming]
    return 2 * q * elem + table


def volume_fill_bytes(q: int, n_sites: int, elem: int = 4) -> int:
    """Algorithmic HBM bytes of writing one site quantity into the render
    volume: per site the q populations and q - 1 table entries read (as in a
    pull step), the packed 8-byte voxel coordinate read and one float
    written."""
    return n_sites * (q * elem + 4 * (q - 1) + 8 + 4)
