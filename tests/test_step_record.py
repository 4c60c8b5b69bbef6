"""The per-step log record (HOTRG.step_record) on CPU: its host arithmetic on what the library
reports (the discarded weight and the relative gap at each cut), with the library's queries
replaced by fixed values."""
import numpy as np
import pytest

from paper_1906_06060_gb300 import HOTRG


def _fake(spectra, dims, axis=3, n=5):
    f = HOTRG.__new__(HOTRG)
    f.observables = lambda instance=0: {"steps": n, "last_axis": axis, "last_ln_c": -0.5,
                                        "lnz_per_site": 0.74, "x_indicator": 1.2}
    f.dims = lambda: tuple(dims)
    f.spectra = lambda step, b, instance=0: np.asarray(spectra.get(b, []), dtype=float)
    return f


def test_step_record_cut_statistics():
    lam = [8.0, 4.0, 2.0, 1.0, 0.5, 0.5, -1e-17]   # a tiny negative value from rounding
    rec = _fake({0: lam, 1: lam[:4], 2: lam}, dims=(4, 4, 5, 3)).step_record()
    assert rec["n"] == 5 and rec["axis"] == 3 and rec["dims"] == [4, 4, 5, 3]
    assert set(rec["cuts"]) == {"0", "1", "2"}      # the step's own axis has no Gram matrix
    c0 = rec["cuts"]["0"]
    total = 8 + 4 + 2 + 1 + 0.5 + 0.5
    assert c0["chi"] == 4 and c0["discarded_weight"] == pytest.approx(1.0 / total)
    assert c0["gap"] == pytest.approx((1.0 - 0.5) / 1.0)
    assert c0["top"][:3] == pytest.approx([1.0, 0.5, 0.25])
    assert rec["cuts"]["1"]["discarded_weight"] == 0.0 and rec["cuts"]["1"]["gap"] is None  # nothing cut
    c2 = rec["cuts"]["2"]
    assert c2["chi"] == 5 and c2["gap"] == pytest.approx(0.0)   # a cut through a degenerate pair


def test_step_record_before_the_first_step():
    rec = _fake({}, dims=(2, 2, 2, 2), axis=-1, n=0).step_record()
    assert rec["n"] == 0 and rec["cuts"] == {}
