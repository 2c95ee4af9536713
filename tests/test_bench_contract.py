"""bench.py's output contract, checked on CPU: the reference arm (the CPU
oracle on a bounded sample) prints one JSON line with the keys a benchmark
line carries, and the roofline helpers do their arithmetic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "0",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_mixed_peak_fraction_arithmetic():
    import bench
    st = {"flops_model": 3.0e12, "flops_model_fp32": 1.0e12}
    r = bench.mixed_peak_frac(st, 1000.0)  # one second
    assert abs(r["fp64_achieved_tflops"] - 2.0) < 1e-12 and abs(r["fp32_achieved_tflops"] - 1.0) < 1e-12
    assert abs(r["combined"] - (2.0 / bench.FP64_PEAK_TFLOPS + 1.0 / bench.FP32_PEAK_TFLOPS)) < 1e-12
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9


def test_fma_probe_compiles_for_sm103a(tmp_path):
    """The probe behind the FP64/FP32 peak figures and the mma.sync rates
    (bench.py --fma-peak / --mma-peak) compiles for sm_103a (it runs only on
    a GPU) and holds the four tensor-core shapes it reports."""
    import shutil
    import bench
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "probe.cu"
    src.write_text(bench.FMA_PROBE_SRC)
    out = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-c", str(src), "-o",
                          str(tmp_path / "probe.o")], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    for shape in ("m8n8k4.row.col.f64", "m16n8k8.row.col.f32.tf32", "m16n8k16.row.col.f32.bf16",
                  "m16n8k32.row.col.s32.s8"):
        assert shape in bench.FMA_PROBE_SRC


def test_kernel_hash_ignores_comments_and_layout():
    """The traffic profile's key changes with the code, not with comments or
    layout; string literals that contain comment markers are code."""
    import bench
    a = 'int a; // note\n/* block\n comment */ const char *s = "x//y/*z*/";\n'
    b = 'int   a;\nconst char *s = "x//y/*z*/";   // other note\n'
    c = 'int a; const char *s = "x//y*/";\n'
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
    assert '"x//y/*z*/"' in bench.code_only(a)


def test_cpu_baseline_counts_sampled_work_only():
    """The CPU baseline times the oracle over a sample of outer shell pairs
    and leaves the per-call setup (Schwarz factors of all pairs) out of the
    rate; on the water trimer the sample is the whole loop (stride 1)."""
    import bench
    import molgen
    import oracle
    p = molgen.problem(0)
    r = bench.cpu_baseline(p, target_s=0.2)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] == oracle.threads()
    assert "not counted" in r["sample"]
    assert bench.oracle_setup_seconds(p) > 0
