"""Host-side logic of bench.py that decides what the JSON line reports (no GPU):

* the source hash that ties a committed ncu summary to the kernel it was taken on follows
  the kernel's own function text (and the headers named with it), not unrelated edits;
* the summary's traffic is reported only while that hash matches, else null;
* the roofline is taken from the kernel family with the largest measured time, with
  achieved = algorithmic cost per launch / measured launch time and frac = achieved / peak.
"""
import os

import pytest

import bench

KERNEL = """template <int OP>
__global__ void __launch_bounds__(256) k_demo(const double *a, double *b) {
  if (a) {
    b[0] = a[0];
  }
}
"""
OTHER = """__global__ void k_other(double *b) { b[0] = 1.0; }
"""


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1610_01265_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "demo.cu").write_text("// header\n" + KERNEL + "\n" + OTHER)
    (csrc / "demo.cuh").write_text("// included\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_function_text_extracts_the_kernel_with_its_template_line():
    text = "// x\n" + KERNEL + OTHER
    got = bench._function_text(text, "k_demo")
    assert got.startswith("template <int OP>") and got.rstrip().endswith("}")
    assert "k_other" not in got and got.count("{") == got.count("}")
    assert bench._function_text(text, "k_missing") == text


def test_source_hash_follows_the_kernel_not_its_neighbours(fake_root):
    src = fake_root / "paper_1610_01265_gb300" / "csrc" / "demo.cu"
    names = ("demo.cu:k_demo", "demo.cuh")
    h0 = bench.kernel_source_hash(names)
    src.write_text(src.read_text().replace("b[0] = 1.0;", "b[0] = 2.0;"))  # another kernel
    assert bench.kernel_source_hash(names) == h0
    src.write_text(src.read_text().replace("b[0] = a[0];", "b[0] = 2 * a[0];"))  # this kernel
    h1 = bench.kernel_source_hash(names)
    assert h1 != h0
    (fake_root / "paper_1610_01265_gb300" / "csrc" / "demo.cuh").write_text("// changed\n")  # its header
    assert bench.kernel_source_hash(names) != h1


def test_traffic_only_while_the_summary_matches_the_source(fake_root):
    names = ("demo.cu:k_demo", "demo.cuh")
    summary = fake_root / "profiles" / "demo.md"
    summary.write_text(f"traffic_bytes_per_launch: 123456789\nkernel_source_sha256_16: {bench.kernel_source_hash(names)}\n")
    assert bench.profiled_traffic("demo.md", names) == 123456789.0
    src = fake_root / "paper_1610_01265_gb300" / "csrc" / "demo.cu"
    src.write_text(src.read_text().replace("b[0] = a[0];", "b[0] = -a[0];"))
    assert bench.profiled_traffic("demo.md", names) is None
    assert bench.profiled_traffic("missing.md", names) is None
    assert bench.profiled_traffic(None, names) is None


def test_roofline_of_takes_the_largest_family_and_its_algorithmic_cost(monkeypatch):
    monkeypatch.setattr(bench, "profiled_traffic", lambda summary, sources: None)
    N = 9437184
    prof = {"conduction": {"spmv": (500.0, 1500), "rkl2_stage": (100.0, 250), "setup": (20.0, 1)},
            "viscosity": {"spmv": (80.0, 550)}}
    roof, per = bench.roofline_of(prof, N, ms_step=1000.0, fp64_peak=1.25, fp64_peak_note="t", hbm_peak=6800.0)
    flop, nbytes = bench.KERNEL_COST[("conduction", "spmv")][:2]
    t = 500.0 / 1500 * 1e-3
    assert roof["kernel"].startswith("spmv (conduction")
    assert roof["achieved"] == pytest.approx(flop * N / t / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1.25)
    assert roof["hbm_achieved_gbs"] == pytest.approx(nbytes * N / t / 1e9)
    assert roof["share_of_step"] == pytest.approx(0.5)
    assert roof["share_of_kernel_time"] == pytest.approx(500.0 / 700.0)
    assert sum(v["share"] for v in per.values()) == pytest.approx(1.0)


def test_committed_summaries_exist_for_every_costed_kernel():
    for (opn, kname), (flop, nbytes, bound, summary, sources) in bench.KERNEL_COST.items():
        assert flop > 0 and nbytes > 0 and bound in ("alu", "hbm")
        if summary:
            assert os.path.exists(os.path.join(bench.ROOT, "profiles", summary)), summary
        for name in sources:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_1610_01265_gb300", "csrc", name.partition(":")[0]))



def test_cpu_sample_mix_is_the_timed_steps_mix():
    """The CPU oracle's sample is weighted by the timed step's own work: its PCG iteration
    counts are the oracle's for this configuration (written by a committed oracle-only
    script) and the stage counts follow from Eq. 5."""
    import json

    import oracle as O

    gold = json.load(open(os.path.join(bench.ROOT, "tests", "golden", "bench_config_iters.json")))
    assert tuple(gold["dims"]) == bench.GRID and tuple(gold["block"]) == bench.BLOCK
    for name in ("jacobi", "bilu0"):
        assert bench.STEP_ITERS[name] == tuple(gold["conduction"][f"{name}_{int(r)}"]["iters"] for r in bench.RATIOS)
    assert bench.STEP_ITERS["visc_jacobi"] == tuple(gold["viscosity"]["jacobi_500"]["iters"])
    assert bench.STEP_ITERS["visc_bilu0"] == tuple(gold["viscosity"]["bilu0_500"]["iters"])
    assert bench.VISC_RATIO == 500.0
    m = bench.step_mix()
    assert m["rkl2_c"] == sum(O.rkl2_stages(r) for r in bench.RATIOS) == 283
    assert m["rkl2_v"] == 3 * O.rkl2_stages(bench.VISC_RATIO)
    passes = sum(m[k] for k in ("rkl2_c", "jacobi_c", "bilu0_c", "rkl2_v", "jacobi_v", "bilu0_v"))
    assert abs(passes - 2601) <= 1  # the GPU step's cell passes (profiled_step_units / cells), to within one iteration
    assert m["factor_c"] == len(bench.RATIOS) and m["factor_v"] == 1
