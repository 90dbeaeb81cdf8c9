"""Domain decomposition plan for running one lattice on several ranks.

HemeLB distributes the sparse site list over MPI ranks and exchanges the
populations that stream across rank boundaries after every step (Section 2,
two-level domain decomposition; Section 3.3.2, lattice data gathered from the
ranks).  This module holds the host-side plan of that decomposition for the
site-list layout of this library:

* partitions are contiguous ranges of the Morton (Z-order) site order, the
  order the device keeps its sites in, sized to hold equal numbers of sites
  (a contiguous range keeps the cut, and so the halo, small);
* the halo of a partition is the set of sites owned by other partitions
  that one of its sites links to (a fluid link in the neighbour table); after
  every step those sites' populations travel from their owners;
* a partition's local problem is its own sites followed by its halo sites,
  with the neighbour table restricted to them: links from own sites keep
  their targets (now local indices), links from a halo site to a site
  outside the local problem become wall links (whatever a halo site
  produces is overwritten by the next exchange).

A local step over own + halo sites reproduces, for the own sites, the step
of the whole lattice exactly: every population arriving at an own site comes
from an own site or from a halo site whose state is an exact copy.

Nothing here touches a GPU; every run in this project uses one GPU, so the
plan is exercised by host tests (the oracle steps the local problems).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np


def _spread3(v: np.ndarray) -> np.ndarray:
    """Interleave the low 21 bits of v with two zero bits between each."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(xyz) -> np.ndarray:
    """Caller indices of the sites sorted along the Z-order curve of their
    coordinates (relative to the bounding box), ties by index."""
    p = np.asarray(xyz, dtype=np.int64).reshape(-1, 3)
    if p.shape[0] == 0:
        return np.empty(0, dtype=np.int64)
    p = p - p.min(axis=0)
    key = _spread3(p[:, 0]) | (_spread3(p[:, 1]) << np.uint64(1)) | (_spread3(p[:, 2]) << np.uint64(2))
    return np.lexsort((np.arange(p.shape[0]), key))


@dataclass
class Partition:
    """One rank's share of the lattice.

    own:   caller indices of the owned sites (a contiguous Morton range).
    halo:  caller indices of the sites of other ranks that own sites link to.
    owner_of_halo: the rank owning each halo site.
    local: own followed by halo (caller indices of the local problem).
    nbr, link: the neighbour table and link flags of the local problem
           ([q][len(local)], local indices; -1 / wall for links that leave it).
    """

    rank: int
    own: np.ndarray
    halo: np.ndarray
    owner_of_halo: np.ndarray
    local: np.ndarray
    nbr: np.ndarray
    link: np.ndarray

    @property
    def n_own(self) -> int:
        return int(self.own.shape[0])


def plan(xyz, nbr, link, k: int) -> List[Partition]:
    """Split the lattice into k Morton ranges of (nearly) equal size and build
    each range's halo and local problem.  nbr and link are the canonical
    tables ([q][n], caller order) of the whole lattice."""
    nbr = np.asarray(nbr)
    link = np.asarray(link)
    q, n = nbr.shape
    if k < 1 or k > max(n, 1):
        raise ValueError("need 1 <= k <= n")
    order = morton_order(xyz)
    bounds = [(n * r) // k for r in range(k + 1)]
    owner = np.empty(n, dtype=np.int64)
    for r in range(k):
        owner[order[bounds[r]:bounds[r + 1]]] = r
    parts = []
    for r in range(k):
        own = np.sort(order[bounds[r]:bounds[r + 1]])
        tgt = nbr[:, own]
        fluid = link[:, own] == 0
        cand = np.unique(tgt[fluid])
        halo = cand[owner[cand] != r]
        local = np.concatenate([own, halo])
        pos = np.full(n, -1, dtype=np.int64)
        pos[local] = np.arange(local.shape[0])
        lnbr = np.empty((q, local.shape[0]), dtype=np.int32)
        llink = np.empty((q, local.shape[0]), dtype=np.uint8)
        for i in range(q):
            t = nbr[i, local]
            lk = link[i, local].copy()
            inside = (lk == 0) & (pos[np.where(t >= 0, t, 0)] >= 0) & (t >= 0)
            lnbr[i] = np.where(inside, pos[np.where(t >= 0, t, 0)], -1)
            # a fluid link that leaves the local problem (from a halo site
            # only) becomes a wall link; wall and iolet links are kept
            llink[i] = np.where((lk == 0) & ~inside, 1, lk)
        if np.any(llink[:, : own.shape[0]] != link[:, own]):
            raise AssertionError("an own site lost a link")  # the halo covers every fluid target
        parts.append(Partition(rank=r, own=own, halo=halo, owner_of_halo=owner[halo], local=local,
                               nbr=lnbr, link=llink))
    return parts


def exchange_lists(parts: Sequence[Partition]):
    """send[r][p]: caller indices of r's own sites that p needs as halo (in
    p's halo order); the same lists give what p receives from r."""
    k = len(parts)
    send = [[np.empty(0, dtype=np.int64) for _ in range(k)] for _ in range(k)]
    for p in parts:
        for r in range(k):
            if r != p.rank:
                send[r][p.rank] = p.halo[p.owner_of_halo == r]
    return send
