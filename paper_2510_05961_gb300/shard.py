"""Sharding independent systems of a batch across GPUs (one process per GPU).

The systems of a batch share nothing, so N GPUs split them with no data-path
collective: each rank builds a ``Batch`` of its own systems and runs it. The
partition is a deterministic longest-processing-time assignment by a cost
model, so every rank computes the same partition without communication.

Cost of one system: its atoms (binning, short range, anterpolation and
interpolation are linear in n) plus the points of all its evaluated grid
levels (restriction, stencils and prolongation are linear in the grid), both
taken from the library's host-side planner (no GPU call).
"""
import ctypes as C

from . import _lib as L


def system_cost(lib, s):
    """Atoms plus grid points of all evaluated levels of one system."""
    P = L.make_params(s.cell, s.pbc, s.h, s.a, s.p, getattr(s, "levels", 0), getattr(s, "grid_override", (0, 0, 0)),
                      0, getattr(s, "qi_mode", 0))
    info = L.PlanInfo()
    L.check(lib.msm_plan_describe(C.byref(P), C.byref(info)))
    pts = 0
    for lv in range(info.ncomp):
        pts += info.n[lv][0] * info.n[lv][1] * info.n[lv][2]
    return int(s.n) + pts


def shard(systems, world, lib=None):
    """Indices of the systems each of `world` ranks evaluates (ascending within a rank).

    Largest cost first, each to the rank with the smallest load so far (ties: the
    lower index, then the lower rank). Every system lands on exactly one rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    lib = lib or L.load()
    cost = [system_cost(lib, s) for s in systems]
    order = sorted(range(len(systems)), key=lambda i: (-cost[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += cost[i]
    return [sorted(p) for p in parts], load
