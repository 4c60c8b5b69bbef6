"""Phase classification from the X^(n) flow (arXiv:1906.06060, Sec. 3, Eq. (x)).

X^(n) = (Tr A^(n))^2 / Tr (A^(n))^2, with A^(n) the coarse-grained tensor traced over the
transverse legs along the step's direction, counts how many singular values of A^(n) share the
largest value. Deep in the disordered phase the flow reaches one dominant value (X -> 1); in the
ordered phase the two symmetry-broken states keep two equal ones (X -> 2). The paper follows
X^(n) until it converges (beyond about 30 steps) and reads the transition temperature off the
change between the two.

The paper gives no convergence threshold. Here a flow counts as converged when its last
`window` values (default 4: one full cycle of the axes, since A^(n) is taken along each step's
own direction) all lie within `tol` of 1 or of 2; otherwise the phase is undetermined (near the
transition the flow converges slowly).

This module is host-side logic on values the library already reports
(`HOTRG.observables(i)["x_indicator"]` after each step).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

DISORDERED = "disordered"
ORDERED = "ordered"
UNDETERMINED = "undetermined"


def classify(x_flow: Sequence[float], tol: float = 0.05, window: int = 4) -> str:
    """Phase of one flow from its X^(n) values (step 1 first)."""
    if window < 1 or tol <= 0:
        raise ValueError("window >= 1 and tol > 0 required")
    tail = [float(x) for x in x_flow][-window:]
    if len(tail) < window or not all(math.isfinite(x) for x in tail):
        return UNDETERMINED
    if all(abs(x - 1.0) <= tol for x in tail):
        return DISORDERED
    if all(abs(x - 2.0) <= tol for x in tail):
        return ORDERED
    return UNDETERMINED


def bracket(betas: Sequence[float], phases: Sequence[str]) -> tuple[float, float] | None:
    """The transition bracket of a scan: for increasing beta, the last disordered point and the
    first ordered point after it, provided every point below is disordered and every point
    above is ordered (undetermined points in between widen the bracket). None if the scan does
    not show one clean change."""
    if len(betas) != len(phases):
        raise ValueError("betas and phases differ in length")
    order = np.argsort(np.asarray(betas, dtype=float), kind="stable")
    b = [float(betas[i]) for i in order]
    p = [phases[i] for i in order]
    dis = [i for i, q in enumerate(p) if q == DISORDERED]
    ordd = [i for i, q in enumerate(p) if q == ORDERED]
    if not dis or not ordd:
        return None
    lo, hi = max(dis), min(ordd)
    if lo >= hi:
        return None
    return b[lo], b[hi]


def x_flow(flow, nsteps: int) -> np.ndarray:
    """Step a HOTRG context `nsteps` times and collect X^(n) after every step.

    Returns an array [nsteps, batch]. Each step synchronises the context's stream (the values
    are read back from the device)."""
    out = np.empty((nsteps, flow.batch))
    for n in range(nsteps):
        flow.step()
        for i in range(flow.batch):
            out[n, i] = flow.observables(i)["x_indicator"]
    return out
