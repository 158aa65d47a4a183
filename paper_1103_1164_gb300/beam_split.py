"""One plan over several ranks, split by beam.

Eq. (1) is a sum over beamlets, and every beamlet belongs to one beam, so a
plan's dose is the sum of the doses of its beams.  Each rank builds a plan of
its share of the beams (the whole density grid, the beams' fluence slices) on
its own GPU, computes that partial dose, and the ranks add the partials.  The
exchange is one all-gather of the V-float partial doses; the partials are then
added in rank order, so every rank gets the same sums in the same order
(deterministic).  The shares are contiguous runs of beams balanced by beamlet
count.

Orchestration only: the dose itself comes from the caller's dose function
(the library's dc_fspb_dose on the rank's GPU).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List

import numpy as np


def beam_shares(beamlets_per_beam: List[int], world: int) -> List[List[int]]:
    """Contiguous runs of beams, one per rank, with beamlet totals as even as
    the beams allow (greedy cut at the running total's 1/world marks).  A rank
    may get no beam when there are fewer beams than ranks."""
    total = float(sum(beamlets_per_beam))
    shares: List[List[int]] = [[] for _ in range(world)]
    acc = 0.0
    for b, n in enumerate(beamlets_per_beam):
        mid = acc + 0.5 * n                      # the beam goes to the rank whose slice holds its middle
        r = min(world - 1, int(mid / total * world)) if total > 0 else 0
        shares[r].append(b)
        acc += n
    return shares


def sub_plan(plan_in, beams: List[int]):
    """The plan restricted to `beams` (same grid, density and model; the
    fluence entries of those beams, in order)."""
    bpb = plan_in.beamlets_per_beam
    first = np.concatenate([[0], np.cumsum(bpb)]).astype(int)
    flu = np.concatenate([plan_in.fluence[first[b]:first[b + 1]] for b in beams]) if beams else \
        np.zeros(0, np.float32)
    return dataclasses.replace(plan_in, beams=[plan_in.beams[b] for b in beams], fluence=flu.astype(np.float32))


def dose_split(plan_in, dose_fn: Callable, rank: int, world: int, all_gather: Callable) -> np.ndarray:
    """The plan's dose [V] from this rank's share of the beams.

    dose_fn(sub_plan) -> [V] partial dose of the rank's beams (zeros if the
    rank has none); all_gather(x) -> list of every rank's x (rank order)."""
    shares = beam_shares(plan_in.beamlets_per_beam, world)
    mine = shares[rank]
    if mine:
        part = np.asarray(dose_fn(sub_plan(plan_in, mine)), np.float64).reshape(-1)
    else:
        part = np.zeros(plan_in.grid.n_voxels)
    parts = all_gather(part)
    out = np.zeros_like(part)
    for p in parts:                              # rank order: the same sums on every rank
        out += p
    return out
