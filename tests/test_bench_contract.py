"""The benchmark's JSON contract on the host: the reference arm (the FP64
oracle timed on the host cores) needs no GPU, so its line is checked here
-- keys, workload and metric shared with the GPU arm, zero transfer bytes,
rank 0 alone printing under a multi-rank launch -- and the warm-up rule."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _bench(*args, env=None):
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=600, env={**os.environ, **(env or {})})


def test_reference_arm_prints_the_contract_line():
    r = _bench("--impl", "reference", "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in KEYS:
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["unit"] == "MLUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 2
    assert line["config"]["workload"] == "fp32_4096x1024_shear_0.05"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]


def test_reference_arm_other_ranks_print_nothing():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3",
               env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_below_three_is_refused():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "2")
    assert r.returncode != 0 and "warmup" in r.stderr


def test_kernel_digest_ignores_comments_only(tmp_path, monkeypatch):
    """The digest that ties a committed profile to the kernel source changes
    with the code, not with its comments or layout."""
    sys.path.insert(0, ROOT)
    import bench
    src = open(bench.KERNEL_SRC, encoding="utf-8").read()
    base = bench.kernel_source_digest()
    p = tmp_path / "k.cu"
    p.write_text("// a new comment\n" + src.replace("\n", "\n\n", 3) + "\n/* trailing\n block */\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(p))
    assert bench.kernel_source_digest() == base
    p.write_text(src.replace("kWaitLimit = 1u << 22", "kWaitLimit = 1u << 21"))
    assert bench.kernel_source_digest() != base


def test_profiled_traffic_follows_the_summary_and_its_digest(tmp_path, monkeypatch):
    """roofline.traffic: the committed summary's back-to-back bytes per step
    times the steps of one launch, with its basis; None (and the reason)
    when the summary is missing, gives no bytes, or was taken on another
    kernel source."""
    sys.path.insert(0, ROOT)
    import bench
    digest = bench.kernel_source_digest()
    p = tmp_path / "summary.md"
    p.write_text(f"# x\n\nkernel source digest: `{digest}` (sha256 ...)\n"
                 "dram bytes per step: 1000 (back to back, 20-step launch)\n")
    monkeypatch.setitem(bench.PROFILE, "fp32", str(p))
    traffic, basis = bench.profiled_traffic("fp32", 20)
    assert traffic == 20000 and basis.startswith("20 steps x 1000")
    p.write_text("kernel source digest: `0123456789abcdef`\ndram bytes per step: 1000 (x)\n")
    traffic, basis = bench.profiled_traffic("fp32", 20)
    assert traffic is None and "changed" in basis
    p.write_text(f"kernel source digest: `{digest}`\n")
    assert bench.profiled_traffic("fp32", 20)[0] is None
    monkeypatch.setitem(bench.PROFILE, "fp32", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic("fp32", 20) == (None, "no committed ncu summary")
    assert bench.profiled_traffic("no such precision", 20) == (None, "no committed ncu summary")


def test_step_launches_of_one_call():
    """One lb_step(h, K) call: a single-step launch for K = 1, else
    multi-step launches of at most max(2, 2^30 / tiles) steps each."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.step_launches(1, 720) == (1, "lbk::sweep_step_kernel")
    assert bench.step_launches(20, 720) == (1, "lbk::sweep_multi_kernel")
    chunk = (1 << 30) // 720
    assert bench.step_launches(chunk + 1, 720) == (2, "lbk::sweep_multi_kernel")
    assert bench.step_launches(5, 1 << 31) == (3, "lbk::sweep_multi_kernel")
