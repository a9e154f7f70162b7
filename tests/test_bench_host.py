"""Host logic of bench.py that the reported roofline depends on (CPU only): a committed ncu summary
supplies `traffic` only while the kernel's definition (and the shared device helpers) is the one it
was captured on, and a capture on a smaller case is scaled by the algorithmic bytes."""
import os
import shutil

import pytest

import bench


def test_kernel_hash_covers_the_definition(tmp_path, monkeypatch):
    src = os.path.join("paper_0811_2518_gb300", "csrc", "solve32.cu")
    h1 = bench.kernel_source_sha(src, "k32_mean")
    assert h1 == bench.kernel_source_sha(src, "k32_mean")  # stable
    assert h1 != bench.kernel_source_sha(src, "k32_joint")  # per kernel
    # a copy of the tree whose k32_mean body differs by one character hashes differently
    root = tmp_path / "r"
    (root / "paper_0811_2518_gb300" / "csrc").mkdir(parents=True)
    for f in ("solve32.cu", "devutil.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_0811_2518_gb300", "csrc", f),
                    root / "paper_0811_2518_gb300" / "csrc" / f)
    p = root / "paper_0811_2518_gb300" / "csrc" / "solve32.cu"
    text = p.read_text()
    i = text.index("k32_mean(Args32 a) {")
    j = text.index("const int t = ctl->round + 1;", i)
    p.write_text(text[:j] + "const int t = ctl->round + 1;  " + text[j + len("const int t = ctl->round + 1;"):])
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_source_sha(src, "k32_mean") != h1


def test_profiled_traffic_follows_the_kernel_hash(tmp_path, monkeypatch):
    src = os.path.join("paper_0811_2518_gb300", "csrc", "solve32.cu")
    sha = bench.kernel_source_sha(src, "k32_mean")
    root = tmp_path / "r"
    shutil.copytree(os.path.join(bench.ROOT, "paper_0811_2518_gb300", "csrc"),
                    root / "paper_0811_2518_gb300" / "csrc")
    (root / "profiles").mkdir()
    summary = ("- kernel_source_sha256: `{}` (definition)\n- dram_bytes_per_launch: 1000\n"
               "- algorithmic_bytes_captured: 500\n")
    (root / "profiles" / "fresh.md").write_text(summary.format(sha))
    (root / "profiles" / "stale.md").write_text(summary.format("0" * 64))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._profiled_traffic("fresh.md", src, "k32_mean") == pytest.approx(1000.0)
    assert bench._profiled_traffic("fresh.md", src, "k32_mean", scale_to=1500) == pytest.approx(3000.0)
    assert bench._profiled_traffic("stale.md", src, "k32_mean") is None
    assert bench._profiled_traffic("missing.md", src, "k32_mean") is None


def test_committed_summaries_parse():
    """Every committed kernel summary names a kernel of the current sources (the hash itself may
    lag a kernel change; bench.py then reports no traffic rather than a stale one)."""
    import re

    for f in sorted(os.listdir(os.path.join(bench.ROOT, "profiles"))):
        text = open(os.path.join(bench.ROOT, "profiles", f)).read()
        m = re.search(r"kernel_source_sha256: `(\w+)` \(definition of `(\w+)` in (\S+)", text)
        if not m:
            continue
        assert len(m.group(1)) == 64
        bench.kernel_source_sha(m.group(3), m.group(2))  # the kernel still exists there


def test_reference_arm_line_and_budget(monkeypatch, capsys):
    """`bench.py --impl reference` prints one JSON line with the contract's keys, and shrinks its
    per-step sample (same generator, smaller n) when warm-up + steps rounds would overrun its budget."""
    import json
    import types

    monkeypatch.setattr(bench, "N_NODES", 1 << 16)
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 1e-3)  # forces the smallest sample
    args = types.SimpleNamespace(steps=3, warmup=1)
    assert bench.run_reference(args, rank=0, world=1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["sample_n"] == 1 << 14
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == (bench.oracle_threads() or 1)
    assert line["cpu_baseline"]["host"]["nproc"] == os.cpu_count()
    assert bench.run_reference(args, rank=1, world=2) == 0  # other ranks exit without work
    assert capsys.readouterr().out == ""
