"""FP64 oracle of beamlet fluence from MLC leaf sequences (fluence.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may use it; the product path never does.  Section 2.3 of
the paper converts each plan's leaf sequences and monitor units into a fluence
map on the beamlet grid; fluence.c states that conversion as the plain
definition (meterset-weighted open area of each beamlet, by polygon clipping in
the (x, meterset) plane).  Sequences come from ``synth.LeafSequence``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import oracle as _o


def _lib():
    L = _o.lib()
    if not getattr(L, "_fluence_ready", False):
        vp, i32, d = C.c_void_p, C.c_int, C.c_double
        L.or_open_area.restype = d
        L.or_open_area.argtypes = [d] * 8
        L.or_leaf_fluence.argtypes = [i32, i32, d, d, d, d, i32, i32, vp, vp, vp, vp, vp, d, vp, i32]
        L._fluence_ready = True
    return L


def open_area(l0, r0, l1, r1, m0, m1, xa, xb) -> float:
    """Area of the quadrilateral (l0, m0), (r0, m0), (r1, m1), (l1, m1) between x = xa and x = xb."""
    return _lib().or_open_area(*(float(v) for v in (l0, r0, l1, r1, m0, m1, xa, xb)))


def leaf_fluence(seq, field_x, field_y, bx, by, threads=None) -> np.ndarray:
    """Fluence [N * M] (beamlet (m, n) at n M + m) of one beam's sequence."""
    M, N = int(round(field_x / bx)), int(round(field_y / by))
    d64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    edges, mu, left, right = d64(seq.edges), d64(seq.mu), d64(seq.left), d64(seq.right)
    jaws = d64(seq.jaws)
    out = np.empty(M * N)
    _lib().or_leaf_fluence(M, N, float(field_x), float(field_y), float(bx), float(by),
                           int(edges.size - 1), int(mu.size), _o._p(edges), _o._p(mu), _o._p(left),
                           _o._p(right), _o._p(jaws), float(seq.transmission), _o._p(out),
                           threads or _o.default_threads())
    return out


def plan_fluence(plan, seqs, threads=None) -> np.ndarray:
    """The plan's fluence vector [B] from one sequence per beam (beam order)."""
    return np.concatenate([leaf_fluence(s, b.field_x, b.field_y, plan.beamlet_x, plan.beamlet_y, threads)
                           for s, b in zip(seqs, plan.beams)])
