"""Write the oracle's expected values for the GPU parity tests (calls only oracle/).

    python tests/golden/make_golden.py

Each file records the FP64 oracle flow of one configuration: per step the axis, bond
dimensions, ln c_n, the ln Z/N estimate, X^(n), the cut gaps and the leading Gram spectra
(normalised by the largest eigenvalue). A flow whose cut splits a degenerate multiplet
(gap < 1e-10) is cut-ambiguous from that step on; the file records the first such step.

The impurity_* files record the impure-tensor estimates after every step
(oracle.hotrg_ref.impurity_flow). The deriv_* files record d(ln Z/N)/d beta and d(ln Z/N)/d h after every step with the isometries
frozen (oracle.hotrg_ref.fixed_isometry_derivatives).

    python tests/golden/make_golden.py [name ...]     # only the named files
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import hotrg_ref as R  # noqa: E402

CONFIGS = {
    # 4D, beta = 0.1497, h = 0, Dcut = 4, 16 steps to 16^4 (the small FP64 configuration)
    "flow_d4_b0.1497_h0_D4_n16": dict(d=4, beta=0.1497, h=0.0, Dcut=4, nsteps=16),
    # same at Dcut = 5: no degenerate multiplet at any cut, so every step is comparable
    "flow_d4_b0.1497_h0_D5_n16": dict(d=4, beta=0.1497, h=0.0, Dcut=5, nsteps=16),
    # with a field (breaks the Z2 symmetry; h = 1e-6 as in the differentiation scans)
    "flow_d4_b0.1497_h1e-6_D4_n8": dict(d=4, beta=0.1497, h=1e-6, Dcut=4, nsteps=8),
    # 2D, Dcut = 8, 40 steps to 2^40 sites
    "flow_d2_b0.3_h0_D8_n40": dict(d=2, beta=0.3, h=0.0, Dcut=8, nsteps=40),
    # the benchmark's configuration (4D, beta = 0.1497, h = 0, Dcut = 10), its first four steps:
    # three warm-up steps and the first steady-state step (bond dimensions 10^4); no cut of these
    # steps splits a degenerate multiplet. Step 4 alone is 2e15 flops (about two hours on eight
    # cores), so this file is written only when named: make_golden.py flow_d4_b0.1497_h0_D10_n4
    "flow_d4_b0.1497_h0_D10_n4": dict(d=4, beta=0.1497, h=0.0, Dcut=10, nsteps=4),
}

# written only when named on the command line (hours of CPU)
ON_REQUEST = {"flow_d4_b0.1497_h0_D10_n4"}

DERIV_CONFIGS = {
    # 4D, Dcut = 5, 8 steps: near the transition at h = 0, and with a field of 0.01
    "deriv_d4_b0.1497_h0_D5_n8": dict(d=4, beta=0.1497, h=0.0, Dcut=5, nsteps=8),
    "deriv_d4_b0.16_h0.01_D5_n8": dict(d=4, beta=0.16, h=0.01, Dcut=5, nsteps=8),
    # the differentiation workload's point (beta = 0.1497, h = 1e-6, Dcut = 10), its first three
    # steps (the third makes every bond 10): no cut of these steps splits a degenerate multiplet
    # (at Dcut = 8 the second step's cut does, so its derivative does not exist there)
    "deriv_d4_b0.1497_h1e-6_D10_n3": dict(d=4, beta=0.1497, h=1e-6, Dcut=10, nsteps=3),
}

IMPURITY_CONFIGS = {
    # impure-tensor estimates <s_i s_j>, <s_i> (Eqs. (energy), (spin)), 4D Dcut = 5, 8 steps
    "impurity_d4_b0.16_h0.01_D5_n8": dict(d=4, beta=0.16, h=0.01, Dcut=5, nsteps=8),
}

AMBIGUOUS_GAP = 1e-10


def flow_record(cfg):
    f = R.run(**cfg)
    steps = []
    first_ambiguous = None
    for n in range(cfg["nsteps"]):
        gaps = {str(b): (None if g == float("inf") else g) for b, g in f.gaps[n].items()}
        if first_ambiguous is None and any(g is not None and g < AMBIGUOUS_GAP for g in gaps.values()):
            first_ambiguous = n + 1
        spec = {}
        for b, lam in f.spectra[n].items():
            top = lam[: cfg["Dcut"] + 2]
            spec[str(b)] = [float(x) for x in (top / lam[0])]
        steps.append(dict(step=n + 1, axis=f.axes[n], dims=list(f.dims[n]), ln_c=f.ln_c[n + 1],
                          lnz=f.lnz[n + 1], x=f.x[n], gaps=gaps, spectra=spec))
    return dict(config=cfg, ln_c0=f.ln_c[0], lnz_final=f.lnz[-1], first_ambiguous_step=first_ambiguous,
                steps=steps, source="oracle/hotrg_ref.py run(), FP64")


def deriv_record(cfg):
    f = R.run(**cfg)
    gaps = [min(g.values()) for g in f.gaps if g]
    db, dh = R.fixed_isometry_derivatives(**cfg)
    fb, fh = R.flow_derivatives(**cfg)
    return dict(config=cfg, lnz=[float(x) for x in f.lnz], dlnz_dbeta=[float(x) for x in db],
                dlnz_dh=[float(x) for x in dh], flow_dlnz_dbeta=[float(x) for x in fb],
                flow_dlnz_dh=[float(x) for x in fh], min_cut_gap=float(min(gaps)),
                source="oracle/hotrg_ref.py fixed_isometry_derivatives() (eps = 1e-3) and "
                       "flow_derivatives() (eps = 1e-4), FP64 central differences, Richardson")


def impurity_record(cfg):
    f = R.impurity_flow(**cfg)
    return dict(config=cfg, nn=[float(x) for x in f.nn], spin=[float(x) for x in f.spin],
                source="oracle/hotrg_ref.py impurity_flow(), FP64")


def main():
    only = set(sys.argv[1:])
    for name, cfg in IMPURITY_CONFIGS.items():
        if only and name not in only:
            continue
        rec = impurity_record(cfg)
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(rec, fh, indent=1)
        print(name, rec["nn"][-1], rec["spin"][-1])
    for name, cfg in DERIV_CONFIGS.items():
        if only and name not in only:
            continue
        rec = deriv_record(cfg)
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(rec, fh, indent=1)
        print(name, rec["dlnz_dbeta"][-1], rec["dlnz_dh"][-1], "min gap", rec["min_cut_gap"])
    for name, cfg in CONFIGS.items():
        if (only and name not in only) or (not only and name in ON_REQUEST):
            continue
        rec = flow_record(cfg)
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(rec, fh, indent=1)
        print(name, rec["lnz_final"], "first ambiguous step:", rec["first_ambiguous_step"])


if __name__ == "__main__":
    main()
