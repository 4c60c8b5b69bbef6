"""Phase classification from the X^(n) flow (Sec. 3, Eq. (x)): the host logic on synthetic flows,
pinned on the oracle against Onsager's exact 2D transition, and the library's batched X^(n)
flows against the oracle's on a GB300."""
import math

import numpy as np
import pytest

from oracle import hotrg_ref as R
from paper_1906_06060_gb300 import phase as PH


def test_classify_reads_the_converged_tail():
    assert PH.classify([1.7, 1.3, 1.02, 1.01, 1.0, 1.0]) == PH.DISORDERED
    assert PH.classify([1.0, 1.4, 1.97, 2.0, 2.01, 2.0]) == PH.ORDERED
    assert PH.classify([1.0, 1.0, 1.0, 1.5]) == PH.UNDETERMINED          # not converged
    assert PH.classify([2.0, 1.0, 2.0, 1.0]) == PH.UNDETERMINED          # oscillating
    assert PH.classify([1.0, 1.0, 1.0]) == PH.UNDETERMINED               # shorter than a cycle
    assert PH.classify([1.0, 1.0, float("nan"), 1.0]) == PH.UNDETERMINED
    assert PH.classify([1.08, 1.08, 1.08, 1.08], tol=0.1) == PH.DISORDERED
    assert PH.classify([1.08, 1.08, 1.08, 1.08], tol=0.05) == PH.UNDETERMINED
    with pytest.raises(ValueError):
        PH.classify([1.0], window=0)


def test_bracket_needs_one_clean_change():
    D, O, U = PH.DISORDERED, PH.ORDERED, PH.UNDETERMINED
    assert PH.bracket([0.1, 0.2, 0.3, 0.4], [D, D, O, O]) == (0.2, 0.3)
    assert PH.bracket([0.4, 0.1, 0.3, 0.2], [O, D, O, D]) == (0.2, 0.3)   # any order of the grid
    assert PH.bracket([0.1, 0.2, 0.3, 0.4], [D, U, U, O]) == (0.1, 0.4)   # widened by undetermined
    assert PH.bracket([0.1, 0.2, 0.3], [D, D, D]) is None
    assert PH.bracket([0.1, 0.2, 0.3, 0.4], [D, O, D, O]) is None         # no single change
    with pytest.raises(ValueError):
        PH.bracket([0.1], [D, O])


def test_x_flow_collects_every_step_and_instance():
    class Fake:
        batch = 2

        def __init__(self):
            self.n = 0

        def step(self):
            self.n += 1

        def observables(self, i):
            return {"x_indicator": 10.0 * self.n + i}

    x = PH.x_flow(Fake(), 3)
    assert x.shape == (3, 2) and x.tolist() == [[10, 11], [20, 21], [30, 31]]


def test_oracle_2d_scan_brackets_onsagers_transition():
    """2D Ising, 40 steps (a 2^20 x 2^20 lattice) at Dcut 8: the bracket of the classified scan
    contains the exact beta_c = ln(1 + sqrt 2) / 2."""
    beta_c = math.log(1.0 + math.sqrt(2.0)) / 2.0
    betas = [0.42, 0.435, 0.44, 0.4415, 0.446, 0.46]
    phases = [PH.classify(R.run(2, b, 0.0, 8, 40).x) for b in betas]
    assert phases[0] == PH.DISORDERED and phases[-1] == PH.ORDERED
    lo, hi = PH.bracket(betas, phases)
    assert lo < beta_c < hi and hi - lo < 0.002


def test_oracle_4d_flows_on_both_sides_of_the_transition():
    """4D at Dcut 4 (24 steps): T = 7.14 is disordered, T = 6.25 ordered; the paper's
    T_c(Dcut = 13) = 6.650365 lies between."""
    assert PH.classify(R.run(4, 0.14, 0.0, 4, 24).x) == PH.DISORDERED
    assert PH.classify(R.run(4, 0.16, 0.0, 4, 24).x) == PH.ORDERED


@pytest.mark.gpu
def test_library_x_flows_classify_like_the_oracle():
    from paper_1906_06060_gb300 import HOTRG
    betas, nsteps = [0.14, 0.16], 24
    with HOTRG(4, betas, 0.0, 4, max_steps=nsteps) as f:
        x = PH.x_flow(f, nsteps)
    for i, b in enumerate(betas):
        ref = R.run(4, b, 0.0, 4, nsteps).x
        np.testing.assert_allclose(x[:2, i], ref[:2], rtol=0, atol=1e-9)   # lossless steps
        assert PH.classify(x[:, i]) == PH.classify(ref) == [PH.DISORDERED, PH.ORDERED][i]
