"""Host-side arithmetic of bench.py (no GPU): the pair count behind the
roofline's algorithmic bytes, the kernel names the roofline reports, and the
rule that a committed DRAM-traffic figure is quoted only while the kernel
source it was captured on is unchanged."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_pairs_per_walk_counts_truncated_windows(bench):
    # brute force: every (center, context) with 0 < |o| <= W inside the walk
    want = sum(1 for p in range(bench.L) for q in range(bench.L) if p != q and abs(p - q) <= bench.WINDOW)
    assert bench._pairs_per_walk() == want == 1490


def test_kernel_names_follow_the_automatic_forms(bench):
    assert bench._sgns_kernel_name(0, "fp32") == "k_sgns_hogwild_hw<128,float,5,false>"
    assert bench._sgns_kernel_name(0, "bf16") == "k_sgns_hogwild_pf<128,bf16,5>"
    assert bench._sgns_kernel_name(3, "fp32") == "k_sgns_hogwild_hw<128,float,5,true>"
    assert bench._sgns_kernel_name(1, "bf16") == "k_sgns_hogwild<128,bf16,8,5>"
    assert bench._sgns_kernel_name(5, "fp32") == "k_sgns_hogwild_bulk<128,5>"


def test_profile_traffic_only_for_the_captured_source(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    h = bench._kernel_source_hash([str(src)])
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "p.md").write_text(f"# x\n\n- sgns.cu + sgns_core.cuh sha256[:16]: `{h}`\n"
                               "- dram_bytes_per_full_launch: 123000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profile_traffic([str(src)], "p.md") == 123000.0
    src.write_text("kernel v2\n")
    assert bench._profile_traffic([str(src)], "p.md") is None
    assert bench._profile_traffic([str(src)], "missing.md") is None


def test_profile_commands_parse(bench, monkeypatch):
    """Every bench.py command quoted in a committed profile summary is one the
    current bench.py accepts (the summaries say how to reproduce them)."""
    import glob
    import re
    import shlex

    cmds = []
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^>&\n`\"]*)", text):
            cmds.append((os.path.basename(path), shlex.split(m.group(1))))
    assert len(cmds) >= 10
    for name, argv in cmds:
        monkeypatch.setattr("sys.argv", ["bench.py"] + argv)
        bench._args()  # argparse exits on an unknown option or value
