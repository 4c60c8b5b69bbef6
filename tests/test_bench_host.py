"""bench.py's host logic on CPU: argument defaults, which contexts run block-sparse, the
workload description, and the committed-profile lookup that feeds roofline.traffic."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def args(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


def test_defaults_name_the_dcut10_flow(monkeypatch):
    a = args(monkeypatch)
    assert (a.dcut, a.precision, a.fp64_steps, a.x6_steps, a.warmup, a.steps) == (10, "fp16x3", 3, 6, 12, 4)
    assert args(monkeypatch, "--workload", "scan").dcut == 8
    assert bench.steady_flops(10) == 2.0e15


def test_block_sparse_only_where_the_structure_holds(monkeypatch):
    assert bench.use_z2(args(monkeypatch))                              # h = 0 flow
    assert bench.use_z2(args(monkeypatch, "--precision", "fp64"))       # FP64 steps too
    assert not bench.use_z2(args(monkeypatch, "--no-z2"))
    assert not bench.use_z2(args(monkeypatch, "--h", "1e-6"))           # field breaks the symmetry
    assert not bench.use_z2(args(monkeypatch, "--workload", "deriv"))   # h-tangent is odd


def test_scan_splits_into_a_block_sparse_and_a_dense_context(monkeypatch):
    a = args(monkeypatch, "--workload", "scan", "--instances", "3")
    betas, hs = bench.instances(a)
    assert len(betas) == 6 and hs == [0.0] * 3 + [1e-5] * 3
    g = bench.groups(a)
    assert [(len(b), z) for b, _, z in g] == [(3, True), (3, False)]
    assert g[0][1] == [0.0] * 3 and g[1][1] == [1e-5] * 3
    assert sorted(g[0][0] + g[1][0]) == sorted(betas)
    cfg = bench.workload_config(a)
    assert cfg["contexts"] == [{"instances": 3, "z2": True}, {"instances": 3, "z2": False}]
    assert cfg["instances"] == 6 and cfg["h"] == [0.0, 1e-5]


def test_workload_config_records_the_timed_steps(monkeypatch):
    cfg = bench.workload_config(args(monkeypatch, "--warmup", "5", "--steps", "2"))
    assert cfg["timed_steps"] == [6, 7] and cfg["Dcut"] == 10 and cfg["z2_block_sparse"]
    assert cfg["parallelism"] == "single GPU" and "workload" in cfg


def _profile(tmp_path, sha, traffic):
    p = tmp_path / "prof.md"
    p.write_text(f"# summary\n\n- gemm_tc_sha={sha}\n- traffic_bytes_per_launch_full={traffic}\n")
    return str(p)


def test_traffic_is_read_only_while_the_kernel_source_is_unchanged(tmp_path, monkeypatch):
    src = tmp_path / "gemm_tc.cu"
    src.write_bytes(b"// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    monkeypatch.setattr(bench, "GEMM_SRC", str(src))
    monkeypatch.setattr(bench, "PROFILE", {True: _profile(tmp_path, sha, "1.2300e+10"),
                                           False: str(tmp_path / "missing.md")})
    assert bench.traffic_from_profile(True, 1) == pytest.approx(1.23e10)  # no cta_group line: single CTAs
    assert bench.traffic_from_profile(True, 2) is None        # counters taken with the other CTA group
    assert bench.traffic_from_profile(False, 1) is None       # no summary
    src.write_bytes(b"// kernel source, changed\n")
    assert bench.traffic_from_profile(True, 1) is None        # counters taken on another kernel


def test_effective_cta_group_follows_the_autotuner_then_the_flag_then_the_default(monkeypatch):
    class A:
        cta_group = 0
    a = A()
    monkeypatch.setattr(bench, "use_z2", lambda _: True)
    assert bench.effective_cta_group(a, [{"kblock": 64, "cta_group": 1}]) == 1
    assert bench.effective_cta_group(a, "off") == 2          # block-sparse default: pairs
    monkeypatch.setattr(bench, "use_z2", lambda _: False)
    assert bench.effective_cta_group(a, []) == 1             # dense default: single CTAs
    a.cta_group = 2
    assert bench.effective_cta_group(a, []) == 2


def test_committed_profiles_parse():
    for z2, path in bench.PROFILE.items():
        with open(path) as fh:
            text = fh.read()
        assert "gemm_tc_sha=" in text and "traffic_bytes_per_launch_full=" in text, path


def test_accuracy_line_reads_the_committed_fp64_reference(monkeypatch, tmp_path):
    """The bench's accuracy line compares its flow's ln Z/N after each step with the FP64 GPU flow
    recorded in the committed accuracy summary (and the oracle's golden, when present)."""
    ref = bench.stored_fp64_reference()
    assert sorted(ref) == list(range(1, 9)) and all(0.7 < v < 1.2 for v in ref.values())
    p = tmp_path / "acc.md"
    p.write_text("# x\n\n- fp64_lnz_step_1 = 1.5\n- fp64_lnz_step_2 = 1.25\n")
    monkeypatch.setattr(bench, "ACCURACY_PROFILE", str(p))
    monkeypatch.setattr(bench, "ORACLE_GOLDEN_D10", str(tmp_path / "missing.json"))
    a = args(monkeypatch)
    acc = bench.accuracy_line(a, [1.5 * (1 + 1e-8), 1.25 * (1 - 2e-8), 1.1])
    assert acc["rel_err_vs_fp64_gpu"]["1"] == pytest.approx(1e-8, rel=1e-6)
    assert acc["rel_err_vs_fp64_gpu"]["2"] == pytest.approx(2e-8, rel=1e-6)
    assert acc["rel_err_vs_oracle"] == {} and acc["lnz_per_site_last"] == 1.1
    assert bench.accuracy_line(args(monkeypatch, "--dcut", "8"), [1.0]) is None   # other configuration


def test_scan_group_is_the_largest_that_fits(monkeypatch):
    class FakeCuda:
        def __init__(self, free):
            self.free = free

        def mem_get_info(self):
            return self.free, self.free

    class FakeTorch:
        def __init__(self, free):
            self.cuda = FakeCuda(free)

    a = args(monkeypatch, "--workload", "scan")
    assert bench.squeeze_group(a, FakeTorch(1e15)) == 64
    assert bench.squeeze_group(a, FakeTorch(1e6)) == 1
    assert bench.squeeze_group(args(monkeypatch, "--workload", "scan", "--group", "4"), FakeTorch(1e6)) == 4
    assert bench.squeeze_group(args(monkeypatch), FakeTorch(1e6)) == 0      # single flow: library default
