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
