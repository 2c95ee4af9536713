"""Benchmark of the J/K build (one step = one fock_build_jk call, i.e. one SCF
iteration's Coulomb + exchange build).  Default workload: the (H2O)64
liquid-density water cluster (1,216 Cartesian functions, 6-31G(d)-shaped
synthetic basis, FP64, Schwarz threshold 1e-10, distance-decaying synthetic
density), the largest single-GPU configuration.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is ERIs/s: symmetry-unique contracted
Cartesian ERIs in quartets passing the Schwarz test, divided by the device
time of the build, summed over ranks (independent replicas, weak scaling).
Extra keys: `mixed` (the same workload in mixed precision), `c20h42` (the
C20H42 alkane in FP64 and mixed precision), `batched` (a batch of TZ-shaped
molecules up to f through fock_build_jk_batched, FP64 and mixed).
The reference arm times the CPU oracle (plain FP64 C with OpenMP) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "J+K build s/iteration and ERIs/s vs FP64/FP32 peak; mixed vs FP64 at 1e-7"
UNIT = "ERI/s"
# FP64 peak derived from the GB300 unit counts and clock: 152 SMs x 2 FP64
# FMA/clk/SM x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 (FFMA) peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--carbons", type=int, default=20, help="alkane length for --config 1 (profiling cases)")
    ap.add_argument("--waters", type=int, default=64, help="water molecules for --config 2 (334: 1,002 atoms)")
    ap.add_argument("--nmol", type=int, default=256, help="molecules of the batched workload (--config 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--warp-scratch", type=int, default=0, help="shared-memory doubles per warp (0 = library default)")
    ap.add_argument("--reg-max-l", type=int, default=0, help="largest total L served by register kernels (0 = default)")
    ap.add_argument("--fp32-cutoff", type=float, default=1e-5, help="mixed leg: FP32 below this quartet bound")
    ap.add_argument("--no-mixed-leg", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="measured per-class-pair schedule (fock_autotune) instead of the built-in rule")
    ap.add_argument("--no-extras", action="store_true", help="skip the c20h42 and batched extra keys")
    ap.add_argument("--k-thresh", type=float, default=5e-6, help="tau* of the decay-bound exchange mode")
    ap.add_argument("--batched-nmol", type=int, default=32, help="molecules of the batched extra key")
    ap.add_argument("--mma-peak", action="store_true",
                    help="measure the mma.sync tensor-core rates (f64, tf32, bf16, s8) on one GPU and exit")
    ap.add_argument("--fma-peak", action="store_true",
                    help="measure the DFMA and FFMA peaks with a register-only FMA probe (built with nvcc) and exit")
    ap.add_argument("--chain-study", default=None, metavar="N1,N2,...",
                    help="J-only / K-only build times of zigzag alkanes C_nH_2n+2 for the listed n, exact and "
                         "decay-bound exchange (one JSON line per n) and exit")
    ap.add_argument("--tune-cache", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                         "paper_2407_21445_gb300", "_build", "tune_cache.json"))
    ap.add_argument("--tune-nmol", type=int, default=2, help="--config 3: molecules the schedule is measured on")
    ap.add_argument("--write-traffic", metavar="NCU_CSV", default=None,
                    help="write profiles/jk_h2o64_traffic.json from an ncu CSV launch list with DRAM bytes "
                         "(TRAFFIC_COMMAND) and exit")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the headline leg (mixed: FP32 below --fp32-cutoff)")
    return ap.parse_args()


def workload_config(p, st, precision="fp64"):
    c = p.meta.get("carbons", 20)
    cfg = {"workload": f"C{c}H{2 * c + 2} zigzag alkane, 6-31G(d)-shaped synthetic basis"
           if p.meta.get("config") == 1 else p.name, "nbf": int(p.nbf), "nshell": int(len(p.basis["l"])),
           "schwarz_thresh": p.tau, "screening": "Schwarz + six-block density (Sec. 3.2)",
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas",
           "precision": precision}
    if st is not None:
        cfg["eris_per_step"] = int(st["eris_schwarz"])
        cfg["quartets_per_step"] = int(st["quartets_schwarz"])
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "jk_h2o64_traffic.json")
TRAFFIC_COMMAND = ("ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                   "--clock-control none -c 400 --csv --log-file launches_c2_fp64.csv python bench.py --config 2 "
                   "--steps 1 --warmup 1 --no-extras --no-mixed-leg --no-cpu-baseline")


def profile_traffic(kernel_src_hash: str):
    """DRAM bytes of one (H2O)64 FP64 build from the committed ncu summary, or
    None when the kernel sources changed since the capture."""
    if not os.path.exists(TRAFFIC_PROFILE):
        return None
    try:
        d = json.load(open(TRAFFIC_PROFILE))
    except Exception:
        return None
    if d.get("kernel_source_sha256") != kernel_src_hash:
        return None
    return d.get("dram_bytes_per_build")


def write_traffic(csv_path: str):
    """DRAM bytes of one build from an ncu --csv launch list (one pass:
    gpu__time_duration.sum, dram__bytes_read.sum, dram__bytes_write.sum): the
    library's launches summed and divided by the number of builds (k_dprep
    launches), recorded with the kernel-source hash they belong to."""
    import csv
    import io
    import re
    rows = [l for l in open(csv_path).read().splitlines() if l.startswith('"')]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1.0, "usecond": 1e3,
             "msecond": 1e6, "second": 1e9}
    per, names = {}, {}
    for r in csv.DictReader(io.StringIO("\n".join(rows))):
        v = float(r["Metric Value"].replace(",", "")) * scale.get(r["Metric Unit"], 1.0)
        per.setdefault(r["ID"], {})[r["Metric Name"]] = v
        names[r["ID"]] = r["Kernel Name"]
    ours = [i for i in per if re.search(r"k_reg|k_jk|k_dprep|k_symmetrize", names[i])]
    builds = max(1, sum(1 for i in ours if "k_dprep" in names[i]))
    rd = sum(per[i].get("dram__bytes_read.sum", 0.0) for i in ours) / builds
    wr = sum(per[i].get("dram__bytes_write.sum", 0.0) for i in ours) / builds
    t = sum(per[i].get("gpu__time_duration.sum", 0.0) for i in ours) / builds
    d = {"kernel_source_sha256": kernel_hash(), "builds": builds, "launches_per_build": len(ours) / builds,
         "dram_bytes_read_per_build": rd, "dram_bytes_write_per_build": wr, "dram_bytes_per_build": rd + wr,
         "serialised_ns_per_build": t, "command": TRAFFIC_COMMAND,
         "note": "ncu's default cache control empties the caches before every launch, so each launch re-reads "
                 "its pair data and tables from DRAM"}
    with open(TRAFFIC_PROFILE, "w") as f:
        json.dump(d, f, indent=1)
    return d


_CODE_TOKENS = re.compile(r"//[^\n]*|/\*.*?\*/|'(?:\\.|[^\\'\n])*'|\"(?:\\.|[^\\\"\n])*\"", re.S)


def code_only(src: str) -> str:
    """C/C++/CUDA source with its comments removed and whitespace runs
    collapsed (string and character literals kept as they are)."""
    out = _CODE_TOKENS.sub(lambda m: " " if m.group(0)[0] == "/" else m.group(0), src)
    return " ".join(out.split())


def kernel_hash():
    """SHA-256 over the library's sources (csrc/, by file name) with comments
    and layout removed: the key of the traffic profile, which holds as long
    as the compiled code is the same."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2407_21445_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(f.encode() + b"\0")
        h.update(code_only(open(os.path.join(d, f), encoding="utf-8").read()).encode())
    return h.hexdigest()


def oracle_setup_seconds(p):
    """Per-call fixed cost of oracle.jk_sample: the Schwarz factors of every
    pair and the rest of its setup, which a full build pays once.  Timed on a
    call whose sample is a single outer shell pair (best of two)."""
    import oracle
    best = float("inf")
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.jk_sample(p.basis, p.D, p.tau, 1 << 30)
        best = min(best, time.perf_counter() - t0)
    return best


def oracle_stride(p, seconds, setup):
    """Stride of oracle.jk_sample (every stride-th outer shell pair) for about
    `seconds` of sampled quartet work per call beyond the per-call setup,
    calibrated on growing samples."""
    import oracle
    stride = 1 << 16
    while True:
        t0 = time.perf_counter()
        oracle.jk_sample(p.basis, p.D, p.tau, stride)
        dt = time.perf_counter() - t0 - setup
        if dt >= 1.0 or stride == 1:
            break
        stride //= 4
    return max(1, int(round(stride * max(dt, 1e-3) / seconds)))


def cpu_baseline(p, target_s=12.0):
    """The oracle as it stands, on every host core, over a sample of outer shell
    pairs (every stride-th) of the same workload; the rate counts the sampled
    quartets' time, not the per-call setup a full build pays only once."""
    import oracle
    setup = oracle_setup_seconds(p)
    stride = oracle_stride(p, target_s, setup)
    t0 = time.perf_counter()
    n = oracle.jk_sample(p.basis, p.D, p.tau, stride)
    dt = time.perf_counter() - t0
    work = max(dt - setup, 1e-9)
    return {"value": n / work, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"every {stride}th outer shell pair of the symmetric quartet loop "
                      f"({n:.4g} Schwarz-passing ERIs in {dt:.1f} s, of which the per-call setup "
                      f"(Schwarz factors of all pairs, paid once by a full build) {setup:.2f} s is not counted)"}


def run_reference(args, rank, world):
    import molgen
    import oracle
    if rank != 0:
        return
    p = molgen.problem(args.config, carbons=args.carbons, waters=args.waters)
    cnt = oracle.count(p.basis, p.D, p.tau)
    setup = oracle_setup_seconds(p)
    # whole run within a few minutes: each step's sampled work plus its setup
    budget = max(0.5, 150.0 / max(1, args.steps + args.warmup) - setup)
    stride = oracle_stride(p, budget, setup)
    for _ in range(args.warmup):
        oracle.jk_sample(p.basis, p.D, p.tau, stride)
    tot_n, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        tot_n += oracle.jk_sample(p.basis, p.D, p.tau, stride)
        tot_t += max(time.perf_counter() - t0 - setup, 1e-9)
    value = tot_n / tot_t
    st = {"eris_schwarz": cnt["eris_schwarz"], "quartets_schwarz": cnt["quartets_schwarz"]}
    cfg = workload_config(p, st)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"every {stride}th outer shell pair per step; the per-call setup "
                                       f"(Schwarz factors of all pairs, {setup:.2f} s, paid once by a full build) "
                                       f"is not counted"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(ms: float, dist, dev) -> float:
    """The slowest rank's time (ms): every rank's replica must finish before
    the whole job has processed world x its units."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def mixed_peak_frac(st, ms):
    """Roofline of the mixed path: the modelled FP64 and FP32 operations each
    over their own pipe's peak; `combined` = the fraction of the build time
    the two pipes would need at peak."""
    t = ms * 1e-3
    f32 = st["flops_model_fp32"]
    f64 = st["flops_model"] - f32
    a64, a32 = f64 / t / 1e12, f32 / t / 1e12
    return {"fp64_achieved_tflops": a64, "fp64_frac": a64 / FP64_PEAK_TFLOPS, "fp32_achieved_tflops": a32,
            "fp32_frac": a32 / FP32_PEAK_TFLOPS, "combined": a64 / FP64_PEAK_TFLOPS + a32 / FP32_PEAK_TFLOPS,
            "peaks_tflops": {"fp64": FP64_PEAK_TFLOPS, "fp32": FP32_PEAK_TFLOPS}}


def tuned(args, fk, bases, Ds, tau, prec):
    """Options for the timed builds: the measured per-class-pair schedule
    (fock_autotune, cached per workload shape and GPU) unless --no-autotune;
    tuning runs before, and outside, every timed region."""
    base = fk.make_opts(precision=prec, fp32_cutoff=args.fp32_cutoff, warp_scratch=args.warp_scratch,
                        reg_max_L=args.reg_max_l)
    if not args.autotune:
        return base, {"source": "built-in rule"}
    from paper_2407_21445_gb300 import autotune
    o, rec = autotune.tuned_opts(bases, Ds, tau, base, cache=args.tune_cache, reps=3)
    return o, {"source": "autotuned" + (" (cached)" if rec["cached"] else ""), "tuned_on_molecules": len(bases),
               "ms_built_in_rule": rec["ms_base"], "ms_measured_schedule": rec["ms_tuned"],
               "kept": "measured schedule" if rec["ms_tuned"] < rec["ms_base"] else "built-in rule",
               "class_pairs_changed": len(rec["schedule"])}


def time_steps(torch, dev, stream, flush, fn, steps, warmup):
    """`warmup` untimed calls, then `steps` calls each bracketed by CUDA events
    on the launching stream, with the L2 flushed before each; ms per call."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s_, e_ in evs:
        flush.zero_()
        s_.record(stream)
        fn()
        e_.record(stream)
    torch.cuda.synchronize(dev)
    return [s_.elapsed_time(e_) for s_, e_ in evs]


def batched_leg(args, fk, torch, dev, stream, flush, nmol, steps, warmup, e2e_steps=0):
    """nmol molecules of uneven size (TZ-shaped basis up to f) per step through
    fock_build_jk_batched, FP64 then mixed precision."""
    import molgen
    probs = molgen.batch_problems(nmol)
    tau = probs[0].tau
    Ds = [torch.tensor(p.D, device=dev) for p in probs]
    Js = [torch.empty_like(d) for d in Ds]
    Ks = [torch.empty_like(d) for d in Ds]
    tunes = {}

    def setup(prec):
        k = max(1, min(args.tune_nmol, len(probs)))
        opts, tunes[prec] = tuned(args, fk, [p.basis for p in probs[:k]], Ds[:k], tau, prec)
        return [fk.JKBuilder(p.basis, tau, opts) for p in probs]

    def run(bs):
        hs = [b.handle for b in bs]
        return time_steps(torch, dev, stream, flush, lambda: fk.fock_build_jk_batched(hs, Ds, tau, Js, Ks), steps,
                          warmup)

    bs = setup(fk.FOCK_FP64)
    stats = [b.stats(p.D) for b, p in zip(bs, probs)]
    eris = sum(s["eris_schwarz"] for s in stats)
    flops = sum(s["flops_model"] for s in stats)
    ms = float(np.mean(run(bs)))
    st = fk.fock_stream_status()
    if st != 0:
        raise SystemExit(f"device status {fk.fock_status_string(st)}")
    Jref = [j.clone() for j in Js]
    Kref = [k.clone() for k in Ks]
    e2e_ms = None
    nbytes = sum(d.numel() * 8 for d in Ds)
    if e2e_steps > 0:
        # pinned host densities in, J and K back to pinned host, every step
        Dh = [torch.tensor(p.D).pin_memory() for p in probs]
        Jh = [torch.empty_like(d).pin_memory() for d in Dh]
        Kh = [torch.empty_like(d).pin_memory() for d in Dh]
        hs = [b.handle for b in bs]
        e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e_s.record(stream)
        for _ in range(e2e_steps):
            for d, h in zip(Ds, Dh):
                d.copy_(h, non_blocking=True)
            fk.fock_build_jk_batched(hs, Ds, tau, Js, Ks)
            for j, k, jh, kh in zip(Js, Ks, Jh, Kh):
                jh.copy_(j, non_blocking=True)
                kh.copy_(k, non_blocking=True)
        e_e.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = e_s.elapsed_time(e_e) / e2e_steps
    for b in bs:
        b.close()
    mbs = setup(fk.FOCK_MIXED)
    mst = [b.stats(p.D) for b, p in zip(mbs, probs)]
    mms = float(np.mean(run(mbs)))
    err = max(max(float((j - jr).abs().max()), float((k - kr).abs().max()))
              for j, k, jr, kr in zip(Js, Ks, Jref, Kref))
    for b in mbs:
        b.close()
    q32 = sum(s["quartets_fp32"] for s in mst)
    q = sum(s["quartets_evaluated"] for s in mst)
    f32 = sum(s["flops_model_fp32"] for s in mst)
    mflops = sum(s["flops_model"] for s in mst)
    nbf = [p.nbf for p in probs]
    achieved = flops / (ms * 1e-3) / 1e12
    return {
        "workload": f"{len(probs)} molecules of 5-40 atoms (water clusters, alkanes, mixtures), TZ-shaped "
                    "synthetic basis up to f, batched build (fock_build_jk_batched, CUDA graph)",
        "molecules": len(probs), "nbf_total": int(sum(nbf)), "nbf_min": int(min(nbf)), "nbf_max": int(max(nbf)),
        "schwarz_thresh": tau, "eris_per_step": int(eris), "steps": steps, "warmup": warmup,
        "fp64": {"ms_per_step": ms, "value": eris / (ms * 1e-3), "unit": UNIT, "achieved_tflops": achieved,
                 "frac_of_fp64_peak": achieved / FP64_PEAK_TFLOPS, "schedule": tunes.get(fk.FOCK_FP64)},
        "mixed": {"ms_per_step": mms, "value": eris / (mms * 1e-3), "unit": UNIT, "speedup_vs_fp64": ms / mms,
                  "fp32_cutoff": args.fp32_cutoff, "max_abs_diff_vs_fp64": err,
                  "fp32_quartet_share": q32 / max(q, 1.0), "fp32_flop_share": f32 / max(mflops, 1.0),
                  "schedule": tunes.get(fk.FOCK_MIXED),
                  "peak_frac": mixed_peak_frac({"flops_model": mflops, "flops_model_fp32": f32}, mms)},
        "_e2e_ms": e2e_ms, "_nbytes": nbytes, "_eris": eris, "_flops": flops,
    }


def run_batched(args, fk, torch, dev, stream, world, rank, dist):
    """--config 3: the batched workload as the headline (FP64), mixed as an
    extra key."""
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if dist:
        dist.barrier()
    with ClockSampler(dev.index) as clk:
        leg = batched_leg(args, fk, torch, dev, stream, flush, args.nmol, args.steps, max(3, args.warmup),
                          e2e_steps=args.steps)
    ms = leg["fp64"]["ms_per_step"]
    ms = max_over_ranks(ms, dist, dev)
    if rank == 0:
        eris, nbytes = leg.pop("_eris"), leg.pop("_nbytes")
        e2e_ms = leg.pop("_e2e_ms")
        flops = leg.pop("_flops")
        achieved = flops / (ms * 1e-3) / 1e12
        cfg = {k: leg[k] for k in ("workload", "molecules", "nbf_total", "nbf_min", "nbf_max", "schwarz_thresh",
                                   "eris_per_step")}
        cfg.update({"l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas",
                    "precision": "fp64", "schedule": leg["fp64"]["schedule"]})
        line = {"metric": METRIC, "value": world * eris / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "s_per_iteration": ms * 1e-3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg,
                "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None},
                "e2e": {"value": world * eris / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(nbytes),
                        "d2h_bytes_per_step": int(2 * nbytes)},
                "mixed": leg["mixed"], "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def alkane_leg(args, fk, torch, dev, stream, flush):
    """C20H42 (384 functions) in FP64 and in mixed precision, W warm-up and K
    timed builds each."""
    import molgen
    p = molgen.problem(1)
    D = torch.tensor(p.D, device=dev, dtype=torch.float64)
    J, K = torch.empty_like(D), torch.empty_like(D)
    out = {"workload": "C20H42 zigzag alkane, 6-31G(d)-shaped synthetic basis, tau=1e-10", "nbf": int(p.nbf),
           "steps": args.steps, "warmup": max(3, args.warmup)}
    ref = None
    for name, prec in (("fp64", fk.FOCK_FP64), ("mixed", fk.FOCK_MIXED)):
        b = fk.JKBuilder(p.basis, p.tau, fk.make_opts(precision=prec, fp32_cutoff=args.fp32_cutoff))
        st = b.stats(p.D)
        ms = float(np.mean(time_steps(torch, dev, stream, flush, lambda: b.build(D, J, K), args.steps,
                                      max(3, args.warmup))))
        leg = {"ms_per_step": ms, "value": st["eris_schwarz"] / (ms * 1e-3), "unit": UNIT}
        if prec == fk.FOCK_FP64:
            ach = st["flops_model"] / (ms * 1e-3) / 1e12
            leg.update(achieved_tflops=ach, frac_of_fp64_peak=ach / FP64_PEAK_TFLOPS)
            ref = (ms, J.clone(), K.clone())
        else:
            leg.update(speedup_vs_fp64=ref[0] / ms,
                       max_abs_diff_vs_fp64=max(float((J - ref[1]).abs().max()), float((K - ref[2]).abs().max())),
                       fp32_flop_share=st["flops_model_fp32"] / max(1.0, st["flops_model"]),
                       peak_frac=mixed_peak_frac(st, ms))
        out[name] = leg
        b.close()
    return out


# Register-only FMA probe: every thread runs NCH independent chains
# x = x * a + b for `iters` iterations and stores their sum (no memory traffic
# in the loop); 3 warm-up launches, 5 timed with CUDA events.
FMA_PROBE_SRC = r"""
#include <cstdio>
#include <cuda_runtime.h>
template <class T, int NCH>
__global__ void k_fma(T *out, int iters, T a, T b) {
  T x[NCH];
#pragma unroll
  for (int i = 0; i < NCH; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) x[i] = x[i] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <class T, int NCH>
void run(int blocks, int threads, int iters) {
  T *d = nullptr;
  if (cudaMalloc(&d, sizeof(T) * blocks * threads) != cudaSuccess) return;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) k_fma<T, NCH><<<blocks, threads>>>(d, iters, (T)0.999, (T)0.001);
  const int reps = 5;
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) k_fma<T, NCH><<<blocks, threads>>>(d, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaFree(d);
  const double flops = 2.0 * NCH * (double)iters * blocks * threads * reps;
  printf("{\"pipe\": \"%s\", \"blocks\": %d, \"threads\": %d, \"chains\": %d, \"iters\": %d, "
         "\"ms_per_launch\": %.4f, \"tflops\": %.4f, \"status\": \"%s\"}\n",
         sizeof(T) == 8 ? "DFMA" : "FFMA", blocks, threads, NCH, iters, ms / reps, flops / (ms * 1e-3) / 1e12,
         cudaGetErrorString(err));
}
// mma.sync probes: every warp runs NCH independent accumulator chains of
// one tensor-core shape (KIND 0: f64 m8n8k4, 1: tf32 m16n8k8 with f32
// accumulation, 2: bf16 m16n8k16 with f32 accumulation, 3: s8 m16n8k32 with
// s32 accumulation), operands in registers.
template <int KIND, int NCH>
__global__ void k_mma(float *out, int iters) {
  const unsigned t = threadIdx.x;
  float s = 0.f;
  if constexpr (KIND == 0) {
    const double a = 1.0 + t * 1e-3, b = 0.5 - t * 1e-4;
    double c[NCH][2];
#pragma unroll
    for (int i = 0; i < NCH; ++i) c[i][0] = c[i][1] = (double)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < NCH; ++i)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                     : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
    }
#pragma unroll
    for (int i = 0; i < NCH; ++i) s += (float)(c[i][0] + c[i][1]);
  } else if constexpr (KIND == 1 || KIND == 2) {
    const unsigned a0 = 0x3f800000u ^ (t << 4), a1 = 0x3f000000u ^ (t << 5), b0 = 0x3e800000u ^ (t << 6),
                   b1 = 0x3f400000u ^ (t << 3);
    float c[NCH][4];
#pragma unroll
    for (int i = 0; i < NCH; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < NCH; ++i) {
        if constexpr (KIND == 1)
          asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                       "{%8, %9}, {%0, %1, %2, %3};"
                       : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                       : "r"(a0), "r"(a1), "r"(a1), "r"(a0), "r"(b0), "r"(b1));
        else
          asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                       "{%8, %9}, {%0, %1, %2, %3};"
                       : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                       : "r"(a0), "r"(a1), "r"(a1), "r"(a0), "r"(b0), "r"(b1));
      }
    }
#pragma unroll
    for (int i = 0; i < NCH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  } else {
    const unsigned a0 = 0x01020304u ^ t, a1 = 0x05060708u ^ (t << 8), b0 = 0x0a0b0c0du ^ (t << 16),
                   b1 = 0x01010101u ^ t;
    int c[NCH][4];
#pragma unroll
    for (int i = 0; i < NCH; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < NCH; ++i)
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                     "{%8, %9}, {%0, %1, %2, %3};"
                     : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
                     : "r"(a0), "r"(a1), "r"(a1), "r"(a0), "r"(b0), "r"(b1));
    }
#pragma unroll
    for (int i = 0; i < NCH; ++i) s += (float)(c[i][0] ^ c[i][1] ^ c[i][2] ^ c[i][3]);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <int KIND, int NCH>
void run_mma(int blocks, int threads, int iters) {
  static const char *names[4] = {"DMMA f64 m8n8k4", "mma tf32 m16n8k8", "mma bf16 m16n8k16", "mma s8 m16n8k32"};
  static const double ops[4] = {2.0 * 8 * 8 * 4, 2.0 * 16 * 8 * 8, 2.0 * 16 * 8 * 16, 2.0 * 16 * 8 * 32};
  float *d = nullptr;
  if (cudaMalloc(&d, sizeof(float) * blocks * threads) != cudaSuccess) return;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) k_mma<KIND, NCH><<<blocks, threads>>>(d, iters);
  const int reps = 5;
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) k_mma<KIND, NCH><<<blocks, threads>>>(d, iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaError_t err = cudaGetLastError();
  cudaFree(d);
  const double warps = (double)blocks * threads / 32;
  const double flops = ops[KIND] * NCH * (double)iters * warps * reps;
  printf("{\"pipe\": \"%s\", \"blocks\": %d, \"threads\": %d, \"chains\": %d, \"iters\": %d, "
         "\"ms_per_launch\": %.4f, \"tflops\": %.4f, \"status\": \"%s\"}\n",
         names[KIND], blocks, threads, NCH, iters, ms / reps, flops / (ms * 1e-3) / 1e12, cudaGetErrorString(err));
}
int main(int argc, char **argv) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const bool mma = argc > 1 && argv[1][0] == 'm';
  if (!mma) {
    run<double, 8>(sms * 8, 256, 20000);
    run<double, 8>(sms * 4, 256, 40000);
    run<double, 16>(sms * 8, 256, 10000);
    run<float, 8>(sms * 8, 256, 400000);
    run<float, 16>(sms * 8, 256, 200000);
    run<float, 8>(sms * 16, 256, 200000);
    return 0;
  }
  run_mma<0, 8>(sms * 8, 128, 4000);
  run_mma<0, 4>(sms * 16, 128, 4000);
  run_mma<1, 8>(sms * 8, 128, 40000);
  run_mma<1, 4>(sms * 16, 128, 40000);
  run_mma<2, 8>(sms * 8, 128, 40000);
  run_mma<2, 4>(sms * 16, 128, 40000);
  run_mma<3, 8>(sms * 8, 128, 20000);
  run_mma<3, 4>(sms * 16, 128, 20000);
  return 0;
}
"""


def fma_peak(which="fma"):
    """Build and run the pipe probe (sm_103a) with nvidia-smi clocks sampled:
    which = "fma" (DFMA / FFMA) or "mma" (mma.sync f64 / tf32 / bf16 / s8)."""
    import shutil
    out_dir = os.path.join(ROOT, "paper_2407_21445_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "fma_probe.cu"), os.path.join(out_dir, "fma_probe")
    with open(src, "w") as f:
        f.write(FMA_PROBE_SRC)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
    with ClockSampler(0) as clk:
        r = subprocess.run([exe, which], capture_output=True, text=True, check=True)
    for line in r.stdout.splitlines():
        print(line)
    print(json.dumps({"clocks": clk.summary()}))


def chain_study(args, fk, torch, dev, stream):
    """Sec. 6.4.1-style scaling study: per alkane length, the device time of a
    J-only build, a K-only build with the exact exchange test and a K-only
    build with the decay-bound test (tau* = --k-thresh), and the decay mode's
    K error against the exact one."""
    import molgen
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for n in [int(x) for x in args.chain_study.split(",")]:
        p = molgen.problem(1, carbons=n)
        D = torch.tensor(p.D, device=dev, dtype=torch.float64)
        ex = fk.JKBuilder(p.basis, p.tau)
        dc = fk.JKBuilder(p.basis, p.tau, fk.make_opts(k_mode=1, k_thresh=args.k_thresh))
        out = {"carbons": n, "nbf": int(p.nbf), "nshell": int(len(p.basis["l"])), "schwarz_thresh": p.tau,
               "k_thresh": args.k_thresh}
        res = {}
        for name, b, parts in (("j", ex, "j"), ("k_exact", ex, "k"), ("k_decay", dc, "k"), ("jk_exact", ex, "jk")):
            ms = time_steps(torch, dev, stream, flush, lambda: b.build(D, parts=parts), args.steps,
                            max(1, args.warmup))
            out[name + "_ms"] = float(np.mean(ms))
            res[name] = b.build(D, parts=parts)
        torch.cuda.synchronize(dev)
        dK = res["k_decay"][1] - res["k_exact"][1]
        out["k_decay_max_abs_err"] = float(dK.abs().max())
        out["k_decay_tr_D_err"] = abs(float((D * dK).sum()))
        H, L, R, _ = dc.decay_bound(D)
        out.update(H=H, Lambda=L, R_mean=float(np.mean(R)))
        st = ex.stats(p.D)
        out["eris_schwarz"] = int(st["eris_schwarz"])
        ex.close()
        dc.close()
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.write_traffic:
        print(json.dumps(write_traffic(args.write_traffic)))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.fma_peak:
        return fma_peak()
    if args.mma_peak:
        return fma_peak("mma")

    import torch

    import molgen
    import paper_2407_21445_gb300 as fk

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    if args.chain_study:
        return chain_study(args, fk, torch, dev, stream)
    if args.config == 3:
        return run_batched(args, fk, torch, dev, stream, world, rank, dist)
    p = molgen.problem(args.config, carbons=args.carbons, waters=args.waters)
    prec = fk.FOCK_MIXED if args.precision == "mixed" else fk.FOCK_FP64
    D = torch.tensor(p.D, device=dev, dtype=torch.float64)
    opts, tune = tuned(args, fk, [p.basis], [D], p.tau, prec)
    builder = fk.JKBuilder(p.basis, p.tau, opts)
    st = builder.stats(p.D)
    nk = fk.fock_kernels_per_build(builder.handle)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(max(3, args.warmup)):
        builder.build(D, J, K)
    torch.cuda.synchronize(dev)
    st_code = fk.fock_stream_status()
    if st_code != 0:
        raise SystemExit(f"device status {fk.fock_status_string(st_code)}")

    # ---- device-timed region ------------------------------------------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        for s, e in evs:
            flush.zero_()
            s.record(stream)
            builder.build(D, J, K)
            e.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in evs]
    tot_ms = float(sum(step_ms))
    tot_ms = max_over_ranks(tot_ms, dist, dev)
    ms = tot_ms / args.steps
    value = world * st["eris_schwarz"] * args.steps / (tot_ms * 1e-3)

    # ---- end-to-end: pinned host D in, J and K back to pinned host ----------
    Dh = torch.tensor(p.D, dtype=torch.float64).pin_memory()
    Jh = torch.empty_like(Dh).pin_memory()
    Kh = torch.empty_like(Dh).pin_memory()
    e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = min(args.steps, 3)  # seconds-long builds: the copies are a small share already
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e_s.record(stream)
    for _ in range(e2e_steps):
        D.copy_(Dh, non_blocking=True)
        builder.build(D, J, K)
        Jh.copy_(J, non_blocking=True)
        Kh.copy_(K, non_blocking=True)
    e_e.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e_s.elapsed_time(e_e)
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e_value = world * st["eris_schwarz"] * e2e_steps / (e2e_ms * 1e-3)
    assert np.isfinite(Jh.numpy()).all() and np.isfinite(Kh.numpy()).all()

    # ---- mixed-precision leg on the same workload (extra key) --------------
    mixed = None
    if not args.no_mixed_leg and args.precision == "fp64":
        mopts, mtune = tuned(args, fk, [p.basis], [D], p.tau, fk.FOCK_MIXED)
        mb = fk.JKBuilder(p.basis, p.tau, mopts)
        mst = mb.stats(p.D)
        builder.build(D, J, K)
        Jm = torch.empty_like(D)
        Km = torch.empty_like(D)
        msteps = min(args.steps, 5)
        mms = float(np.mean(time_steps(torch, dev, stream, flush, lambda: mb.build(D, Jm, Km), msteps, 3)))
        err = max(float((Jm - J).abs().max()), float((Km - K).abs().max()))
        trd = abs(float((D * (2 * Jm - Km)).sum() - (D * (2 * J - K)).sum()))
        mixed = {"ms_per_step": mms, "value": st["eris_schwarz"] / (mms * 1e-3), "unit": UNIT,
                 "speedup_vs_fp64": ms / mms, "fp32_cutoff": args.fp32_cutoff,
                 "max_abs_diff_vs_fp64": err, "trace_diff_vs_fp64": trd,
                 "fp32_quartet_share": mst["quartets_fp32"] / max(1.0, mst["quartets_evaluated"]),
                 "fp32_flop_share": mst["flops_model_fp32"] / max(1.0, mst["flops_model"]), "schedule": mtune,
                 "peak_frac": mixed_peak_frac(mst, mms), "steps": msteps, "warmup": 3}
        mb.close()

    # ---- extra keys: C20H42 (FP64 and mixed) and a TZ batch up to f ---------
    extras = {}
    if not args.no_extras and args.config == 2 and world == 1:
        extras["c20h42"] = alkane_leg(args, fk, torch, dev, stream, flush)
        bl = batched_leg(args, fk, torch, dev, stream, flush, args.batched_nmol, 1, 1)
        extras["batched"] = {k: v for k, v in bl.items() if not k.startswith("_")}

    if rank == 0:
        achieved = st["flops_model"] / (ms * 1e-3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "s_per_iteration": ms * 1e-3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic", "config": dict(workload_config(p, st, args.precision), schedule=tune),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": profile_traffic(kernel_hash()) if args.config == 2 else None,
                         "peak_note": "FP64 pipe, 152 SMs x 2 FMA/clk x 2.07 GHz = 1.2586 TFLOP/s (DFMA probe "
                                      "1.256, profiles/fp64_fp32_peak.md); achieved = modelled FP64 flops of the "
                                      "evaluated quartets / device time of the whole build (ERI kernels > 99.9 %)",
                         "traffic_note": "DRAM bytes of one FP64 build's launches (ncu, 1 pass, caches emptied "
                                         "before each launch: the pair data and tables are re-read per launch); "
                                         "algorithmic bytes D + J + K = 3 N^2 x 8 B"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(D.numel() * 8),
                    "d2h_bytes_per_step": int(2 * D.numel() * 8), "steps": e2e_steps},
            "gpu_launches": int(nk * args.steps),
            "mixed": mixed,
            "clocks": clk.summary(),
            "work": {k: st[k] for k in ("quartets_evaluated", "eris_evaluated", "prim_quartets",
                                        "flops_model", "prim_pairs", "pairs")},
        }
        line.update(extras)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
