"""Benchmark: microseconds per reciprocal-space SPME evaluation on GB300 (65536 atoms, 64^3, p = 4).

One step = one full evaluation (bin, spread, forward FFT, influence multiply with energy / virial, inverse
FFT, force interpolation) of the 65536-atom water-like box on one of 1000 jittered position frames that
are resident in HBM (786 MB, larger than L2), replayed from per-frame CUDA graphs. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one process per GPU (under torchrun; without it, bench.py starts torchrun itself). The
single-system headline runs as N independent replicas; the batched and served legs shard their systems
across the ranks. There is no data-path collective, only barriers and a max over ranks around the timed
regions. --impl reference times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "us per PME eval (65536 atoms, 64^3, p=4)"
UNIT = "us/eval"
WORKLOAD = ("65536-atom water-like box (21844 triplets + 2 ion pairs), cubic 86.9 A, 64^3 mesh, p=4, beta=0.34/A, "
            "1000 jittered frames N(0,0.01 A)")
PAPER_US = 206.0  # 4 x Stratix 10, same workload size (context; the paper's own hardware)
N_FRAMES = 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, batch, serving and CPU baseline legs")
    ap.add_argument("--legs", default="", help="comma list of extra legs to run alone (batched, serving, large, "
                                               "profile); skips the headline (profile: a short fixed sequence "
                                               "for ncu captures)")
    ap.add_argument("--write-traffic", default="", metavar="NCU_CSV",
                    help="no GPU work: read an ncu --csv log of dram__bytes_read.sum / dram__bytes_write.sum for "
                         "the six stage kernels of one 64^3 evaluation and write profiles/dram_bytes.json for "
                         "the roofline's traffic field (tied to the current kernel sources)")
    return ap.parse_args()


TRAFFIC_SOURCES = ["paper_2009_12617_gb300/csrc/common.cuh", "paper_2009_12617_gb300/csrc/fft.cuh",
                   "paper_2009_12617_gb300/csrc/stages.cuh", "paper_2009_12617_gb300/csrc/kernels.h",
                   "paper_2009_12617_gb300/csrc/kernels.cu", "paper_2009_12617_gb300/csrc/pdl.cuh"]
STAGE_OF_KERNEL = (("k_bin", "bin"), ("k_spread", "spread"), ("k_fwd", "fft_fwd"), ("k_conv", "influence"),
                   ("k_inv", "fft_inv"), ("k_gather", "gather"))


def write_traffic(csv_path: str) -> None:
    """Mean DRAM read + write bytes per launch of each stage kernel from an ncu --csv metrics log, written to
    profiles/dram_bytes.json with the hash of the kernel sources they were taken from."""
    import csv
    import hashlib

    per_launch = {}
    with open(csv_path, newline="") as f:
        rows = [r for r in csv.reader(f) if r]
    hdr_i = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
    hdr = rows[hdr_i]
    col = {k: hdr.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    for r in rows[hdr_i + 1:]:
        if len(r) < len(hdr) or not r[col["Metric Name"]].startswith("dram__bytes_"):
            continue
        stage = next((st for k, st in STAGE_OF_KERNEL if k in r[col["Kernel Name"]]), None)
        if stage is None:
            continue
        key = (stage, r[col["ID"]])
        v = float(r[col["Metric Value"]].replace(",", "")) * scale.get(r[col["Metric Unit"]], 1.0)
        per_launch[key] = per_launch.get(key, 0.0) + v
    by_stage = {}
    for (stage, _), v in per_launch.items():
        by_stage.setdefault(stage, []).append(v)
    sha = hashlib.sha256(b"".join(open(os.path.join(ROOT, p), "rb").read() for p in TRAFFIC_SOURCES)).hexdigest()
    rec = {"what": "dram__bytes_read.sum + dram__bytes_write.sum per launch of each stage kernel (mean over the "
                   "captured launches), from " + os.path.basename(csv_path) + "; valid only while the kernel "
                   "sources hash to source_sha256",
           "source_files": TRAFFIC_SOURCES, "source_sha256": sha,
           "launches": {st: len(v) for st, v in by_stage.items()},
           "bytes_per_launch": {st: int(round(sum(v) / len(v))) for st, v in by_stage.items()}}
    with open(os.path.join(ROOT, "profiles", "dram_bytes.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec["bytes_per_launch"]))


# ---------------------------------------------------------------------------------------------------------
# distributed plumbing (replicas only)


class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def shard(items: list, rank: int, world: int) -> list:
    """Round-robin share of independent systems for one rank (batched / served work needs no collective)."""
    return items[rank::world]


def gather_all(dist: "Dist", obj):
    """Every rank's obj as a list (rank order); [obj] on one process."""
    if not dist.pg:
        return [obj]
    out = [None] * dist.world
    dist.pg.all_gather_object(out, obj)
    return out


def cpu_model() -> str:
    """CPU model name (lscpu, else /proc/cpuinfo; Arm part numbers of the Neoverse cores named)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    parts = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1", "0xd49": "Neoverse-N2"}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
                if ln.lower().startswith("cpu part"):
                    v = ln.split(":", 1)[1].strip()
                    return parts.get(v, f"Arm part {v}")
    except OSError:
        pass
    return os.uname().machine


def errors_vs_oracle(E, V, F, sysobj, threads: int | None = None) -> dict:
    """Relative energy, RMS force and virial error of one GPU result against the FP64 oracle."""
    import oracle

    oracle.build()
    oracle.set_threads(threads or os.cpu_count() or 1)
    try:
        r = oracle.spme(sysobj.pos.astype(np.float64), sysobj.q.astype(np.float64), sysobj.K, sysobj.p, sysobj.beta,
                        sysobj.box)
    finally:
        oracle.set_threads(1)
    F = np.asarray(F, dtype=np.float64)
    return {"rel_energy_error": float(abs(E - r["energy"]) / abs(r["energy"])),
            "rms_force_error": float(np.sqrt(np.mean((F - r["forces"]) ** 2) / np.mean(r["forces"] ** 2))),
            "rel_virial_error": float(np.max(np.abs(np.asarray(V) - r["virial"])) / np.max(np.abs(r["virial"]))),
            "tolerance": {"rel_energy": 1e-6, "rms_force": 1e-5, "rel_virial": 1e-5}}


# ---------------------------------------------------------------------------------------------------------
# clock sampling during the timed regions


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []  # (time, sm_mhz, max_mhz, reasons)
        self.windows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = [n for n, v in zip(names, parts[5:9]) if v.lower() == "active"]
            self.samples.append((time.time(), sm, mx, reasons))

    def window(self, t0, t1):
        self.windows.append((t0, t1))

    def summary(self):
        if self.proc:
            self.proc.terminate()
        inside = [s for s in self.samples if any(a - 0.05 <= s[0] <= b + 0.05 for a, b in self.windows)]
        use = inside or self.samples
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = sorted({r for s in use for r in s[3]})
        return {"sm_mhz": statistics.median(s[1] for s in use), "sm_max_mhz": max(s[2] for s in use),
                "reasons": reasons, "samples": len(use), "in_timed_region": len(inside)}


# ---------------------------------------------------------------------------------------------------------
# algorithmic bytes per stage launch (minimal data each stage must move)


def stage_bytes(n: int, K, p: int) -> dict:
    """Algorithmic bytes per stage launch: what each step of the method must read and write at the least,
    whatever the implementation (the library's own bucket records and its wider influence table are not
    counted). Per atom: 12 B position + 4 B charge in, 12 B force out; per mesh point: 8 B int64 charge mesh,
    4 B potential; per half-spectrum point: 8 B complex FP32 in and out, 8 B FP64 influence value."""
    K1, K2, K3 = K
    mesh = K1 * K2 * K3
    half = K1 * K2 * (K3 // 2 + 1)
    return {
        "bin": n * (16 + 16),                # position + charge in; mesh base (3 int32) + order key out
        "spread": n * 16 + mesh * 8,         # atoms in, int64 charge mesh out
        "fft_fwd": mesh * 8 + half * 8,      # int64 mesh in, complex half spectrum out
        "influence": half * (8 + 8 + 8),     # spectrum in, FP64 influence value in, spectrum out
        "fft_inv": half * 8 + mesh * 4,      # spectrum in, phi out
        "gather": mesh * 4 + n * (16 + 12),  # phi in, atoms in, forces out
    }


def spread_atomics(n: int, p: int) -> int:
    """32-bit shared-memory atomics the spreading stage needs: n p^3 contributions, each a 64-bit fixed-point
    addition made of two native 32-bit atomics (this part has no native 64-bit shared-memory atomicAdd)."""
    return 2 * n * p ** 3


def measure_atomic_peaks(dev) -> dict:
    """Conflict-free shared-memory int32 atomicAdd and global int64 reduction throughput of this GPU, each
    probe kernel timed alone with CUDA events on its stream (best of 5 after warm-up)."""
    import torch

    from paper_2009_12617_gb300 import pme

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream(dev)
    out = {}
    for kind, name, ctas, rounds, nbytes in ((0, "smem_i32_atomics_per_s", 4 * sms, 256, 4 * 4 * sms),
                                             (1, "global_i64_red_per_s", 4 * sms, 32, 4 << 20)):
        buf = torch.zeros(nbytes // 4, dtype=torch.int32, device=dev)
        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 0.0
        with torch.cuda.stream(stream):
            for rep in range(8):
                st.record(stream)
                ops = pme.pme_probe_launch(kind, ctas, rounds, buf, stream)
                en.record(stream)
                en.synchronize()
                if rep >= 3:
                    best = max(best, ops / (st.elapsed_time(en) * 1e-3))
        out[name] = best
    out["how"] = ("probe kernels of this library (pme_probe_launch): 4 CTAs of 512 threads per SM, 8 independent "
                  "atomics per thread per round; smem: distinct words, one bank per lane; global: a 4 MiB "
                  "L2-resident buffer, consecutive 64-bit words per warp")
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measure_l2_gbs(dev) -> float:
    """L2-resident copy bandwidth (read + write bytes per second) of this GPU, measured here: a 24 MiB
    device-to-device copy (48 MiB touched, well inside the 129 MB L2) repeated back to back, best of 5."""
    import torch

    n = 24 * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(5):
        for _ in range(5):
            b.copy_(a)
        st.record()
        for _ in range(50):
            b.copy_(a)
        en.record()
        en.synchronize()
        best = max(best, 50 * 2 * n * 4 / (st.elapsed_time(en) * 1e-3) / 1e9)
    return best


def traffic_record(stage: str):
    """ncu DRAM bytes per launch of the stage's kernel from the committed capture summary, or None when the
    kernel sources changed since the counters were taken (or no capture exists)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "dram_bytes.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        sha = hashlib.sha256(b"".join(open(os.path.join(ROOT, p), "rb").read() for p in TRAFFIC_SOURCES)).hexdigest()
        if sha != rec["source_sha256"]:
            return None
        return rec["bytes_per_launch"].get(stage)
    except (OSError, ValueError, KeyError):
        return None


# ---------------------------------------------------------------------------------------------------------
# our implementation


def run_ours(args, dist: Dist):
    import torch

    from paper_2009_12617_gb300 import build as libbuild
    from paper_2009_12617_gb300 import pme
    from paper_2009_12617_gb300 import workloads as wl

    libbuild.build_library()
    pme.load_library()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    sampler = ClockSampler(dist.local)

    s = wl.headline_system(seed=2)
    L = float(s.box[0, 0])
    # 1000 successive jittered frames (N(0, 0.01 A) random walk), all resident in HBM
    frames_np = np.empty((N_FRAMES, s.n, 3), np.float32)
    cur = s.pos
    for f in range(N_FRAMES):
        frames_np[f] = cur
        cur = wl.jitter(cur, L, 1000 + dist.rank, f)
    frames = torch.from_numpy(frames_np).to(dev)
    SAMPLE = 500  # the frame whose result is checked against the oracle
    sample_pos = frames_np[SAMPLE].copy()
    del frames_np
    q = torch.from_numpy(s.q).to(dev)
    forces = torch.empty((s.n, 3), dtype=torch.float32, device=dev)
    ev = torch.zeros(7, dtype=torch.float64, device=dev)

    stream = torch.cuda.Stream(dev)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    pme.pme_reserve(plan, s.n)

    # one CUDA graph per frame (6 kernel nodes each)
    graphs = []
    with torch.cuda.stream(stream):
        for f in range(N_FRAMES):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                pme.pme_enqueue(plan, frames[f], q, forces, ev)
            graphs.append(g)
        for i in range(max(args.warmup, 3)):
            graphs[i % N_FRAMES].replay()
    pme.pme_sync(plan)

    # ten consecutive frames per graph, so evaluations inside a graph keep their programmatic launch edges
    G = 10
    graphs10 = []
    with torch.cuda.stream(stream):
        for c in range(N_FRAMES // G):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for f in range(c * G, (c + 1) * G):
                    pme.pme_enqueue(plan, frames[f], q, forces, ev)
            graphs10.append(g)
        for i in range(max(args.warmup // G, 1)):
            graphs10[i % len(graphs10)].replay()
    pme.pme_sync(plan)

    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    dist.barrier()
    t0 = time.time()
    with torch.cuda.stream(stream):
        start.record(stream)
        nfull, rest = divmod(args.steps, G)
        for i in range(nfull):  # exactly args.steps evaluations: full ten-frame graphs, then single frames
            graphs10[i % len(graphs10)].replay()
        for i in range(rest):
            graphs[(nfull * G + i) % N_FRAMES].replay()
        end.record(stream)
    torch.cuda.synchronize(dev)
    t1 = time.time()
    dist.barrier()
    sampler.window(t0, t1)
    pme.pme_sync(plan)
    ms_local = start.elapsed_time(end)
    ms = dist.max(ms_local)
    value = 1000.0 * ms / (args.steps * dist.world)  # us per evaluation, whole job
    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 6), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": round(value / PAPER_US, 6), "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "l2": "inputs larger than L2: 1000 distinct position frames (786 MB) cycled; mesh and tables "
                         "stay L2-resident by design",
                   "launch": "CUDA graphs of ten consecutive frames (60 kernels, programmatic dependent launch "
                             "released at CTA exit, the influence stage's successor right after its wait), "
                             "replayed back to back; exactly `steps` evaluations",
                   "evals_per_s": round(1e6 / value, 1)},
        "gpu_launches": 6 * args.steps,
    }
    del graphs10
    if dist.rank != 0:
        return None, sampler, plan, locals()

    # eager (no graph) launches, for context
    with torch.cuda.stream(stream):
        for i in range(20):
            pme.pme_enqueue(plan, frames[i], q, forces, ev)
        torch.cuda.synchronize(dev)
        ne = min(args.steps, 2000)
        t0 = time.time()
        start.record(stream)
        for i in range(ne):
            pme.pme_enqueue(plan, frames[i % N_FRAMES], q, forces, ev)
        end.record(stream)
        torch.cuda.synchronize(dev)
        sampler.window(t0, time.time())
    result["config"]["eager_us_per_eval"] = round(1000.0 * start.elapsed_time(end) / ne, 3)

    # launch-mode sweep: plain launches and programmatic dependent launch triggered at kernel start or right
    # after each kernel's own wait, same frames, fresh graphs (the headline above uses the default, triggered
    # at CTA exit except after the influence stage's wait)
    modes = {}
    for mode in (0, 1, 3):
        pme.pme_set_launch_mode(mode)
        gm = []
        with torch.cuda.stream(stream):
            for f in range(100):
                gg = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gg, stream=stream):
                    pme.pme_enqueue(plan, frames[f], q, forces, ev)
                gm.append(gg)
            for i in range(20):
                gm[i % 100].replay()
            torch.cuda.synchronize(dev)
            nm = min(args.steps, 2000)
            start.record(stream)
            for i in range(nm):
                gm[i % 100].replay()
            end.record(stream)
            torch.cuda.synchronize(dev)
        name = {0: "plain_launch", 1: "pdl_early", 3: "pdl_after_wait"}[mode]
        modes[f"{name}_us_per_eval"] = round(1000.0 * start.elapsed_time(end) / nm, 3)
        del gm
    pme.pme_set_launch_mode(2)  # the library default
    # slab-split sweep: the forward / inverse slab stages on 2 or 4 CTAs per slab (thread-block clusters;
    # the default, one CTA per slab, is the headline)
    for cs in (2, 4):
        pme.pme_set_slab_split(cs)
        gm = []
        with torch.cuda.stream(stream):
            for f in range(100):
                gg = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gg, stream=stream):
                    pme.pme_enqueue(plan, frames[f], q, forces, ev)
                gm.append(gg)
            for i in range(20):
                gm[i % 100].replay()
            torch.cuda.synchronize(dev)
            nm = min(args.steps, 2000)
            start.record(stream)
            for i in range(nm):
                gm[i % 100].replay()
            end.record(stream)
            torch.cuda.synchronize(dev)
        modes[f"slab_split_{cs}_us_per_eval"] = round(1000.0 * start.elapsed_time(end) / nm, 3)
        del gm
    pme.pme_set_slab_split(1)  # the library default
    pme.pme_sync(plan)
    result["config"].update(modes)

    # the same evaluation through the batch API with one system (a graph of its grouped stage chain),
    # frame 0 repeated
    bt = pme.pme_batch_create([plan], [s.n], stream=stream)
    try:
        evb = torch.zeros((1, 7), dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(10):
                pme.pme_batch_enqueue(bt, frames[0], q, forces, evb)
            pme.pme_batch_sync(bt)
            nb = min(args.steps, 2000)
            start.record(stream)
            for _ in range(nb):
                pme.pme_batch_enqueue(bt, frames[0], q, forces, evb)
            end.record(stream)
            torch.cuda.synchronize(dev)
            pme.pme_batch_sync(bt)
        result["config"]["batch_api_single_us_per_eval"] = round(1000.0 * start.elapsed_time(end) / nb, 3)
    finally:
        pme.pme_batch_destroy(bt)

    # per-stage kernel time (CUDA events around each kernel, same stream) for the roofline
    stage_us = pme.pme_profile_stages(plan, frames[0], q, forces, reps=200)
    result["stage_us"] = {k: round(v, 3) for k, v in stage_us.items()}
    # Each isolated time includes that kernel's own launch and drain, so they sum to more than one pipelined
    # evaluation; the shares below scale them onto the measured step.
    tot_iso = sum(stage_us.values())
    result["stage_us_share_of_step"] = {k: round(v / tot_iso * value, 3) for k, v in stage_us.items()}
    sb = stage_bytes(s.n, s.K, s.p)
    dom = max(stage_us, key=stage_us.get)
    peak, src = measured_peaks()
    atom = measure_atomic_peaks(dev)
    result["atomic_peaks"] = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in atom.items()}
    achieved_b = sb[dom] / (stage_us[dom] * 1e-6) / 1e9
    traffic = traffic_record(dom)
    hbm_line = {"kernel": dom, "bound": "hbm", "achieved": round(achieved_b, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved_b / peak, 4), "traffic": traffic,
                "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)", "algorithmic_bytes": sb[dom],
                "kernel_us": round(stage_us[dom], 3)}
    if dom == "spread":
        # spreading is bound by its shared-memory atomics: n p^3 64-bit additions (two 32-bit atomics each)
        na = spread_atomics(s.n, s.p)
        rate = na / (stage_us[dom] * 1e-6)
        result["roofline"] = {"kernel": dom, "bound": "atomic", "achieved": round(rate, 1),
                              "peak": round(atom["smem_i32_atomics_per_s"], 1), "unit": "atomic/s",
                              "frac": round(rate / atom["smem_i32_atomics_per_s"], 4), "traffic": traffic,
                              "peak_source": "measured in this run: conflict-free shared-memory int32 atomicAdd "
                                             "probe (atomic_peaks)",
                              "algorithmic_atomics": na, "kernel_us": round(stage_us[dom], 3),
                              "frac_in_step": round(na / (result["stage_us_share_of_step"][dom] * 1e-6)
                                                    / atom["smem_i32_atomics_per_s"], 4)}
        result["roofline_hbm"] = hbm_line
    else:
        result["roofline"] = hbm_line
    # The meshes stay in L2 between stages, so L2 bandwidth is the other ceiling: per stage (its algorithmic
    # bytes over its own launch time) and for the whole evaluation (all stages' bytes over the pipelined time
    # per evaluation), against an L2-resident copy measured here.
    l2 = measure_l2_gbs(dev)
    tot = sum(sb.values())
    result["roofline_l2"] = {
        "bound": "l2", "unit": "GB/s", "peak": round(l2, 1),
        "peak_source": "measured here: L2-resident 24 MiB device copy, read + write bytes",
        "evaluation": {"algorithmic_bytes": tot, "achieved": round(tot / (result["value"] * 1e-6) / 1e9, 1),
                       "frac": round(tot / (result["value"] * 1e-6) / 1e9 / l2, 4)},
        "stages": {k: {"algorithmic_bytes": sb[k], "kernel_us": round(stage_us[k], 3),
                       "achieved": round(sb[k] / (stage_us[k] * 1e-6) / 1e9, 1),
                       "frac_l2": round(sb[k] / (stage_us[k] * 1e-6) / 1e9 / l2, 4),
                       "frac_hbm": round(sb[k] / (stage_us[k] * 1e-6) / 1e9 / peak, 4)} for k in sb},
    }
    # oracle error of one evaluated frame (frame 500 of the trajectory, through the synchronous entry point)
    with torch.cuda.stream(stream):
        pos_s = torch.from_numpy(sample_pos).to(dev)
        E_s, V_s = pme.pme_compute(plan, pos_s, q, forces)
        F_s = forces.cpu().numpy()
    result["accuracy"] = {"sample": f"frame {SAMPLE} of the jittered trajectory",
                          **errors_vs_oracle(E_s, V_s, F_s, wl.System(sample_pos, s.q, s.box, s.K, s.p, s.beta))}

    # cuFFT, for comparison only (never part of the library): a 64^3 real-to-complex and complex-to-real
    # transform pair of torch.fft with an elementwise multiply between them, against this library's transform
    # and influence stages
    x = torch.randn(s.K, device=dev)
    tab = torch.rand((s.K[0], s.K[1], s.K[2] // 2 + 1), device=dev)
    with torch.cuda.stream(stream):
        for _ in range(20):
            y = torch.fft.irfftn(torch.fft.rfftn(x) * tab, s=s.K)
        nr = 500
        start.record(stream)
        for _ in range(nr):
            y = torch.fft.irfftn(torch.fft.rfftn(x) * tab, s=s.K)
        end.record(stream)
        torch.cuda.synchronize(dev)
    result["cufft_comparison"] = {
        "rfftn_multiply_irfftn_us": round(1000.0 * start.elapsed_time(end) / nr, 3),
        "ours_fwd_influence_inv_us_isolated": round(stage_us["fft_fwd"] + stage_us["influence"] + stage_us["fft_inv"], 3),
        "ours_fwd_influence_inv_us_share_of_step": round(sum(result["stage_us_share_of_step"][k]
                                                             for k in ("fft_fwd", "influence", "fft_inv")), 3),
        "note": "torch.fft (cuFFT) on the same GPU, FP32, 64^3, eager launches; ours includes the energy and virial "
                "reduction and the int64 mesh conversion; comparison only"}
    del y, x, tab
    return result, sampler, plan, locals()


INFLIGHT = 3  # host-array steps the end-to-end loop keeps in flight


def run_e2e(pme, plan, s, steps: int):
    """End to end through the library's host-array calls on page-locked buffers, every step: positions and
    charges move host -> device (read by the binning kernel over the CPU-GPU link), the evaluation runs, and
    forces, energy and virial move device -> host (written by the library's copy kernel).
    value: pme_enqueue_host with three steps in flight (the host waits for step i - 3's ticket, reads its
    result and enqueues step i), host clock over all steps; host_writes_positions_us: the same with the host copying the
    positions of each step into page-locked memory first; synchronous: pme_compute_host, one call and one wait
    per step."""
    import torch

    stream = torch.cuda.Stream()
    L = float(s.box[0, 0])
    frames = [s.pos.astype(np.float32)]
    for f in range(3):
        frames.append(wl_jitter(frames[-1], L, 900, f))

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype).pin_memory().numpy()

    # four page-locked position frames (prepared before the timed region), one charge array, three
    # force/result sets: step i reads frame i % 4 and writes set i % 3
    P_frames = [pinned((s.n, 3), torch.float32) for _ in frames]
    for P, fr in zip(P_frames, frames):
        P[:] = fr
    Q = pinned(s.n, torch.float32)
    Q[:] = s.q
    outs = [(pinned((s.n, 3), torch.float32), pinned(8, torch.float64)) for _ in range(INFLIGHT)]
    e2e_plan = pme.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    try:
        def run(nsteps, host_writes):
            """host_writes: the host copies step i's frame into a working position array of its slot before
            enqueueing (as an integrator writing its new positions would), instead of cycling prepared frames."""
            tickets = [0] * INFLIGHT
            energy = 0.0
            for i in range(nsteps + INFLIGHT):
                slot = i % INFLIGHT
                if i >= INFLIGHT:
                    pme.pme_host_wait(e2e_plan, tickets[slot])
                    R = outs[slot][1]
                    if R[7] != 0.0:
                        raise RuntimeError(f"device status {R[7]} in step {i - INFLIGHT}")
                    energy += R[0]  # the step's result, read on the host
                if i >= nsteps:
                    continue
                F, R = outs[slot]
                if host_writes:
                    P = P_frames[slot]
                    P[:] = frames[i % len(frames)]
                else:
                    P = P_frames[i % len(P_frames)]
                tickets[slot] = pme.pme_enqueue_host(e2e_plan, P, Q, F, R)
            return energy

        run(10, False)  # records the argument sets' graphs
        t0 = time.perf_counter()
        run(steps, False)
        dt = time.perf_counter() - t0
        t_end = time.time()
        run(10, True)
        t0 = time.perf_counter()
        run(steps, True)
        dt_w = time.perf_counter() - t0
        # device time of the same steps enqueued back to back (CUDA events on the plan stream, no host
        # waits): what the two-in-flight loop converges to when the host keeps ahead
        nd = min(steps, 2000)
        pme.pme_sync(e2e_plan)
        t0 = time.perf_counter()
        for i in range(nd):
            F, R = outs[i % INFLIGHT]
            t = pme.pme_enqueue_host(e2e_plan, P_frames[i % len(P_frames)], Q, F, R)
        pme.pme_host_wait(e2e_plan, t)
        dev_us = 1e6 * (time.perf_counter() - t0) / nd
    finally:
        pme.pme_destroy(e2e_plan)
    # synchronous, for comparison
    pos_h = torch.empty((s.n, 3), dtype=torch.float32).pin_memory()
    q_h = torch.empty(s.n, dtype=torch.float32).pin_memory()
    f_h = torch.empty((s.n, 3), dtype=torch.float32).pin_memory()
    pos_h.numpy()[:] = s.pos
    q_h.numpy()[:] = s.q
    P, Q, F = pos_h.numpy(), q_h.numpy(), f_h.numpy()
    for _ in range(5):
        pme.pme_compute_host(plan, P, Q, F)
    t1 = time.perf_counter()
    for _ in range(steps):
        pme.pme_compute_host(plan, P, Q, F)
    dts = time.perf_counter() - t1
    return {"value": round(1e6 * dt / steps, 3), "unit": UNIT, "h2d_bytes_per_step": s.n * 16,
            "d2h_bytes_per_step": s.n * 12 + 8 * 8, "steps": steps,
            "how": "pme_enqueue_host with three steps in flight on page-locked arrays (pme_host_wait for step "
                   "i-3's ticket, read its energy and status, enqueue step i on prepared position frame i % 4), "
                   "host clock",
            "back_to_back_us_per_step": round(dev_us, 3),
            "back_to_back_how": "the same steps enqueued without waiting (results overwritten), host clock from "
                                "the first enqueue to the last ticket's completion: the device-side rate",
            "host_writes_positions_us": round(1e6 * dt_w / steps, 3),
            "host_writes_how": "the same, the host copying each step's 786 KB of positions into the slot's "
                               "page-locked array before enqueueing it",
            "synchronous_us": round(1e6 * dts / steps, 3),
            "synchronous_how": "pme_compute_host per step (one call and one wait), host clock"}, \
        (t_end - dt, t_end)


def wl_jitter(pos, L, seed, step):
    from paper_2009_12617_gb300 import workloads as wl

    return wl.jitter(pos, L, seed, step).astype(np.float32)


def cpu_baseline(target_seconds: float = 12.0):
    """The FP64 oracle as it stands, timed on full evaluations of the headline workload: single-threaded
    (the reported value), then across all host cores (its OpenMP loops), plus the numpy-FFT FP64 context
    baseline. Median of the runs; table set-up excluded from the numpy figure, included in the oracle's
    (the oracle recomputes its tables every call)."""
    import oracle
    from oracle import numpy_spme
    from paper_2009_12617_gb300 import workloads as wl

    oracle.build()
    s = wl.headline_system(seed=2)
    pos, q = s.pos.astype(np.float64), s.q.astype(np.float64)
    nproc = os.cpu_count() or 1

    def timed(fn, budget, cap=10):
        times, t_start = [], time.perf_counter()
        while True:
            t0 = time.perf_counter()
            fn()
            times.append(time.perf_counter() - t0)
            if time.perf_counter() - t_start > budget or len(times) >= cap:
                return 1e6 * statistics.median(times), len(times)

    oracle.set_threads(1)
    v1, n1 = timed(lambda: oracle.spme(pos, q, s.K, s.p, s.beta, s.box), target_seconds)
    used = oracle.set_threads(nproc)
    try:
        vall, nall = timed(lambda: oracle.spme(pos, q, s.K, s.p, s.beta, s.box), target_seconds / 2)
    finally:
        oracle.set_threads(1)
    plan = numpy_spme.Plan(s.K, s.p, s.beta, s.box)
    vnp, nnp = timed(lambda: plan.evaluate(pos, q), target_seconds / 2)
    return {"value": round(v1, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n1} full evaluations of the 65536-atom 64^3 p=4 box, single thread (median)",
            "cpu": cpu_model(), "nproc": nproc,
            "all_cores": {"value": round(vall, 1), "unit": UNIT, "cores": used, "kind": "oracle",
                          "sample": f"{nall} full evaluations, OpenMP over {used} threads (median)"},
            "numpy_fft_fp64": {"value": round(vnp, 1), "unit": UNIT, "cores": 1, "kind": "context baseline",
                               "sample": f"{nnp} evaluations with numpy's pocketfft in FP64, tables precomputed "
                                         "(median); not the oracle"}}


def run_reference(args, dist: Dist):
    """The reference arm: the FP64 oracle, single-threaded, one full evaluation of the headline box per step
    (W warm-up steps, then K timed steps, capped near two minutes of work)."""
    if dist.rank != 0:
        return
    import oracle
    from paper_2009_12617_gb300 import workloads as wl

    oracle.build()
    oracle.set_threads(1)
    s = wl.headline_system(seed=2)
    pos, q = s.pos.astype(np.float64), s.q.astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(max(1, args.warmup)):
        oracle.spme(pos, q, s.K, s.p, s.beta, s.box)
    t_one = (time.perf_counter() - t0) / max(1, args.warmup)
    executed = max(1, min(args.steps, int(150.0 / max(t_one, 1e-3))))
    times = []
    for i in range(executed):
        t0 = time.perf_counter()
        oracle.spme(pos, q, s.K, s.p, s.beta, s.box)
        times.append(time.perf_counter() - t0)
    v = 1e6 * statistics.mean(times)
    sample = (f"{executed} of {args.steps} requested steps timed, each one full FP64 oracle evaluation of the "
              f"65536-atom 64^3 p=4 box (frame 0), single thread, after {max(1, args.warmup)} warm-up steps")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": dist.world,
            "steps": executed, "warmup": max(1, args.warmup), "ms_per_step": round(v / 1000.0, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": round(v / PAPER_US, 3), "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def spawn_ranks(args) -> int:
    """--gpus N > 1 outside torchrun: run this command again under torchrun with N processes."""
    import socket

    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.write_traffic:
        write_traffic(args.write_traffic)
        return
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args))
    dist = Dist()
    if dist.world != args.gpus and dist.rank == 0:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE {dist.world}; using {dist.world} ranks", file=sys.stderr)
    try:
        if args.impl == "reference":
            run_reference(args, dist)
            return
        if args.legs:
            import torch

            from paper_2009_12617_gb300 import build as libbuild
            from paper_2009_12617_gb300 import pme

            libbuild.build_library()
            pme.load_library()
            torch.cuda.set_device(dist.local)
            sampler = ClockSampler(dist.local)
            out = {}
            table = {"batched": leg_batched, "serving": leg_serving, "large": leg_large, "profile": leg_profile,
                     "slab": leg_slab}
            for name in args.legs.split(","):
                out.update(table[name](args, sampler, dist))
            out["clocks"] = sampler.summary()
            if dist.rank == 0:
                print(json.dumps(out), flush=True)
            return
        result, sampler, plan, ctx = run_ours(args, dist)
        from paper_2009_12617_gb300 import pme

        if not args.no_extras:
            if dist.rank == 0:
                e2e, win = run_e2e(pme, plan, ctx["s"], steps=max(20, min(args.steps // 20, 500)))
                sampler.window(*win)
                result["e2e"] = e2e
            for extra in _extras():
                if extra is leg_large and dist.rank != 0:
                    continue
                try:
                    out = extra(args, sampler, dist)
                    if dist.rank == 0:
                        result.update(out)
                except Exception as exc:  # an extra leg failing must not hide the headline number
                    if dist.rank == 0:
                        result.setdefault("errors", []).append(f"{extra.__name__}: {exc}")
            if dist.rank == 0:
                result["cpu_baseline"] = cpu_baseline()
        if dist.rank == 0:
            result["clocks"] = sampler.summary()
            print(json.dumps(result), flush=True)
        else:
            sampler.summary()
        pme.pme_destroy(plan)
    finally:
        dist.close()


def _time_batch(pme, b, pos, q, F, ev, stream, reps, sampler, dist=None):
    """ms per batch evaluation: warm-up, then reps graph replays bracketed by CUDA events on the batch stream
    (and, across ranks, by barriers with the max taken)."""
    import torch

    st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(3):
            pme.pme_batch_enqueue(b, pos, q, F, ev)
        pme.pme_batch_sync(b)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.time()
        st.record(stream)
        for _ in range(reps):
            pme.pme_batch_enqueue(b, pos, q, F, ev)
        en.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler.window(t0, time.time())
        pme.pme_batch_sync(b)
    ms = st.elapsed_time(en) / reps
    return dist.max(ms) if dist else ms


def leg_batched(args, sampler, dist):
    """64 uneven water-like systems (atom counts log-uniform 1024..32768, meshes 32..64), sharded across the
    ranks, evaluated through the batch API (one graph per step: grouped stage launches, the mesh-shape groups
    in parallel; and, for comparison, the persistent work-list kernel), against one launch sequence per
    system (eager, and replayed from a graph). One system's result is checked against the oracle."""
    import torch

    from paper_2009_12617_gb300 import pme
    from paper_2009_12617_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    all_systems = wl.batch_systems(64, seed=4)
    systems = shard(all_systems, dist.rank, dist.world)
    stream = torch.cuda.Stream(dev)
    plans = [pme.pme_create(s.K, s.p, s.beta, s.box, stream=stream) for s in systems]
    ns = [s.n for s in systems]
    pos = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(dev)
    q = torch.from_numpy(np.concatenate([s.q for s in systems])).to(dev)
    F = torch.empty_like(pos)
    ev = torch.zeros((len(systems), 7), dtype=torch.float64, device=dev)
    offs = np.concatenate([[0], np.cumsum(ns)])
    b = pme.pme_batch_create(plans, ns, stream=stream)
    st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    out = {}
    try:
        t_batch = _time_batch(pme, b, pos, q, F, ev, stream, reps, sampler, dist)  # ms per batch, max over ranks
        Fb, evb = F.clone(), ev.clone()
        pme.pme_batch_set_strategy(b, pme.PME_BATCH_PERSISTENT)
        t_pers = _time_batch(pme, b, pos, q, F, ev, stream, reps, sampler, dist)
        same_pers = bool(torch.equal(F, Fb) and torch.equal(ev, evb))
        pme.pme_batch_set_strategy(b, pme.PME_BATCH_AUTO)
        with torch.cuda.stream(stream):
            # one launch sequence per system, same stream
            for i, pl in enumerate(plans):
                pme.pme_reserve(pl, ns[i])
            views = [(pos[offs[i]:offs[i + 1]], q[offs[i]:offs[i + 1]], F[offs[i]:offs[i + 1]], ev[i]) for i in range(len(plans))]
            for i, pl in enumerate(plans):
                pme.pme_enqueue(pl, *views[i])
            torch.cuda.synchronize(dev)
            st.record(stream)
            for _ in range(reps):
                for i, pl in enumerate(plans):
                    pme.pme_enqueue(pl, *views[i])
            en.record(stream)
            torch.cuda.synchronize(dev)
            t_eager = dist.max(st.elapsed_time(en) / reps)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for i, pl in enumerate(plans):
                    pme.pme_enqueue(pl, *views[i])
            g.replay()
            torch.cuda.synchronize(dev)
            st.record(stream)
            for _ in range(reps):
                g.replay()
            en.record(stream)
            torch.cuda.synchronize(dev)
            t_graph = dist.max(st.elapsed_time(en) / reps)
            for pl in plans:
                pme.pme_sync(pl)
        same = bool(torch.equal(F, Fb) and torch.equal(ev, evb))
        # oracle error of the batch's result for one system (the largest of this rank's share)
        k = int(np.argmax(ns))
        acc = errors_vs_oracle(float(evb[k, 0]), evb[k, 1:].cpu().numpy(), Fb[offs[k]:offs[k + 1]].cpu().numpy(),
                               systems[k])
        nsys, atoms = len(all_systems), int(sum(s.n for s in all_systems))
        alg = sum(sum(stage_bytes(s.n, s.K, s.p).values()) for s in all_systems)
        peak, src = measured_peaks()
        achieved = alg / (t_batch * 1e-3) / 1e9
        out = {"batched": {
            "workload": "64 water-like boxes, N log-uniform in [1024, 32768] (seed 4), 0.1 atoms/A^3, K in {32,40,48,64} "
                        "by 1.4 A spacing, p=4; per step one CUDA graph: systems grouped by mesh shape, one launch "
                        "per stage per group, the groups as parallel branches",
            "systems": nsys, "atoms": atoms, "meshes": sorted({s.K[0] for s in all_systems}), "ranks": dist.world,
            "evals_per_s": round(nsys / (t_batch * 1e-3), 1), "us_per_batch": round(t_batch * 1e3, 2),
            "atom_evals_per_s": round(atoms / (t_batch * 1e-3), 1),
            "persistent_work_list": {"evals_per_s": round(nsys / (t_pers * 1e-3), 1),
                                     "us_per_batch": round(t_pers * 1e3, 2), "bit_identical_to_grouped": same_pers},
            "one_system_per_launch": {"eager_evals_per_s": round(nsys / (t_eager * 1e-3), 1),
                                      "graph_evals_per_s": round(nsys / (t_graph * 1e-3), 1)},
            "speedup_vs_graph_of_single_launches": round(t_graph / t_batch, 3),
            "bit_identical_to_single": same,
            "accuracy": {"sample": f"system {dist.rank + k * dist.world} ({systems[k].n} atoms, {systems[k].K[0]}^3), "
                                   "batch result", **acc},
            "gpu_launches_per_step": 2 + 6 * len({(s.K, s.p) for s in systems}),
            "roofline": {"kernel": "all grouped stage launches of one step (64 systems)", "bound": "hbm",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "algorithmic_bytes": int(alg),
                         "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)"}}}
    finally:
        pme.pme_batch_destroy(b)
        for pl in plans:
            pme.pme_destroy(pl)
    return out


def serving_stream(n_req: int, rank: int, world: int):
    """The served request stream (Poisson arrivals at 20k/s, seed 5; 90% over the 64 batch systems, 10% over
    8 headline systems: global pool indices 0..71) and this rank's part of it: the pool indices it owns
    (round robin), and the arrival times and local pool indices of the requests for those systems."""
    rng = np.random.Generator(np.random.PCG64(5))
    gaps = rng.exponential(1.0 / 20000.0, n_req)
    arrival_all = np.cumsum(gaps)
    which_all = np.where(rng.random(n_req) < 0.9, rng.integers(0, 64, n_req), 64 + rng.integers(0, 8, n_req))
    mine = shard(list(range(72)), rank, world)
    local = {g: i for i, g in enumerate(mine)}
    keep = np.array([int(w) in local for w in which_all])
    which = np.array([local[int(w)] for w in which_all[keep]], dtype=np.int64)
    return arrival_all, which_all, mine, arrival_all[keep], which


def leg_serving(args, sampler, dist, n_req: int = 4000):
    """Poisson arrivals (20k requests/s, seed 5) drawing 90% from 64 config-4 systems and 10% from 8
    65536-atom / 64^3 systems, all with resident plans; every request uses a freshly jittered frame. The
    server admits by a 40 GB device budget and 128 slots; the comparison serves the same stream one system
    per launch, synchronously, in arrival order. Across ranks the systems are sharded and each rank serves
    the requests for its own systems; one served result is checked against the oracle."""
    import collections

    import torch

    from paper_2009_12617_gb300 import pme
    from paper_2009_12617_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    small = wl.batch_systems(64, seed=4)
    big = [wl.headline_system(seed=10 + i) for i in range(8)]
    arrival_all, which_all, mine, arrival, which = serving_stream(n_req, dist.rank, dist.world)
    pool = [(small + big)[g] for g in mine]
    plans = [pme.pme_create(s.K, s.p, s.beta, s.box) for s in pool]
    NF, NBUF = 2, 4
    frames, qs, outs = [], [], []
    for i, s in enumerate(pool):
        L = float(s.box[0, 0])
        f1 = wl.jitter(s.pos, L, 500 + mine[i], 0)
        frames.append([torch.from_numpy(s.pos).to(dev), torch.from_numpy(f1).to(dev)])
        qs.append(torch.from_numpy(s.q).to(dev))
        outs.append([torch.empty((s.n, 3), dtype=torch.float32, device=dev) for _ in range(NBUF)])
        pme.pme_reserve(plans[i], s.n)
    n_all, n_req = n_req, len(which)
    srv = pme.pme_server_create(40 * (1 << 30), 128)
    lat = np.zeros(n_req)
    uses = collections.Counter()
    try:
        # warm every plan once through the server
        for i in range(len(pool)):
            t = pme.pme_submit(srv, plans[i], frames[i][0], qs[i], outs[i][0])
            pme.pme_poll(srv, t, block=True)
        inflight = collections.deque()
        busy_bufs = collections.Counter()
        done = 0
        nxt = 0
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        while done < n_req:
            now = time.perf_counter() - t0
            while nxt < n_req and arrival[nxt] <= now:
                i = int(which[nxt])
                if busy_bufs[i] >= NBUF:
                    break
                k = uses[i]
                t = pme.pme_submit(srv, plans[i], frames[i][k % NF], qs[i], outs[i][k % NBUF])
                if t is None:  # PME_EAGAIN: all slots busy; retry after completions
                    break
                uses[i] += 1
                busy_bufs[i] += 1
                inflight.append((nxt, i, t))
                nxt += 1
            # every in-flight ticket is polled (completions need not come in submission order); the loop
            # spins rather than sleeps, as a timed sleep would round up to tens of microseconds
            still = collections.deque()
            for r, i, t in inflight:
                if pme.pme_poll(srv, t, block=False) == pme.PME_OK:
                    lat[r] = (time.perf_counter() - t0) - arrival[r]
                    busy_bufs[i] -= 1
                    done += 1
                else:
                    still.append((r, i, t))
            inflight = still
        elapsed = time.perf_counter() - t0
        sampler.window(time.time() - elapsed, time.time())
        stats = pme.pme_server_stats(srv)
        # one served result against the oracle: a 65536-atom system if this rank has one, frame 0
        k = max(range(len(pool)), key=lambda i: pool[i].n)
        Fk = torch.full_like(frames[k][0], float("nan"))
        t = pme.pme_submit(srv, plans[k], frames[k][0], qs[k], Fk)
        pme.pme_poll(srv, t, block=True)
        acc = errors_vs_oracle(t.energy.value, np.array(t.virial[:]), Fk.cpu().numpy(), pool[k])
    finally:
        pme.pme_server_destroy(srv)
    atoms = np.array([pool[i].n for i in which])
    # the same stream, one system per launch, synchronous, in arrival order
    lat1 = np.zeros(n_req)
    for i in range(len(pool)):
        pme.pme_compute(plans[i], frames[i][0], qs[i], outs[i][0])
    t0 = time.perf_counter()
    for r in range(n_req):
        while time.perf_counter() - t0 < arrival[r]:
            pass
        i = int(which[r])
        pme.pme_compute(plans[i], frames[i][r % NF], qs[i], outs[i][0])
        lat1[r] = (time.perf_counter() - t0) - arrival[r]
    elapsed1 = time.perf_counter() - t0
    for pl in plans:
        pme.pme_destroy(pl)
    parts = gather_all(dist, (lat.tolist(), lat1.tolist(), float(elapsed), float(elapsed1), int(atoms.sum()),
                              stats["p50_us"], stats["p99_us"], stats["waves"]))
    lat = np.concatenate([np.array(x[0]) for x in parts])
    lat1 = np.concatenate([np.array(x[1]) for x in parts])
    elapsed, elapsed1 = max(x[2] for x in parts), max(x[3] for x in parts)
    atoms = np.array([sum(x[4] for x in parts)])
    n_req = n_all
    if dist.world > 1:  # server-side percentiles: the worst rank's
        stats = {"p50_us": max(x[5] for x in parts), "p99_us": max(x[6] for x in parts),
                 "waves": sum(x[7] for x in parts)}
    arrival = arrival_all
    return {"serving": {
        "workload": "Poisson arrivals 20k req/s (seed 5), 90% from 64 config-4 boxes, 10% from 8 65536-atom 64^3 boxes, "
                    "resident plans, jittered frames, budget 40 GB, 128 slots",
        "requests": n_req, "offered_req_per_s": round(n_req / arrival[-1], 1),
        "throughput_req_per_s": round(n_req / elapsed, 1), "atom_evals_per_s": round(atoms.sum() / elapsed, 1),
        "p50_us": round(1e6 * float(np.percentile(lat, 50)), 2), "p99_us": round(1e6 * float(np.percentile(lat, 99)), 2),
        "latency_from": "request arrival time to completion seen by the client", "ranks": dist.world,
        "accuracy": {"sample": f"one served request on a {pool[k].n}-atom system, frame 0", **acc},
        "server_p50_us": round(stats["p50_us"], 2), "server_p99_us": round(stats["p99_us"], 2),
        "waves": stats["waves"],
        "one_system_per_launch": {"throughput_req_per_s": round(n_req / elapsed1, 1),
                                  "p50_us": round(1e6 * float(np.percentile(lat1, 50)), 2),
                                  "p99_us": round(1e6 * float(np.percentile(lat1, 99)), 2)}}}


def leg_large(args, sampler, dist=None):
    """Precision study at the largest mesh: 262144 water-like atoms, 137.9 A, 128^3, p = 6. For each influence
    path (FP32 register FFTs along k1; the same transforms as split-BF16 matrix products on the tensor cores):
    time per evaluation (CUDA graph replays), per-stage times, and the energy / RMS-force / virial error
    against the FP64 oracle on the same inputs."""
    import torch

    import oracle
    from paper_2009_12617_gb300 import pme
    from paper_2009_12617_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    s = wl.large_system(seed=3)
    stream = torch.cuda.Stream(dev)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        ref = oracle.spme(s.pos.astype(np.float64), s.q.astype(np.float64), s.K, s.p, s.beta, s.box)
    finally:
        oracle.set_threads(1)

    def errs(E, V, F):
        F = np.asarray(F, dtype=np.float64)
        return {"rel_energy_error": float(abs(E - ref["energy"]) / abs(ref["energy"])),
                "rms_force_error": float(np.sqrt(np.mean((F - ref["forces"]) ** 2) / np.mean(ref["forces"] ** 2))),
                "rel_virial_error": float(np.max(np.abs(np.asarray(V) - ref["virial"])) / np.max(np.abs(ref["virial"])))}

    out = {}
    try:
        pos = torch.from_numpy(s.pos).to(dev)
        q = torch.from_numpy(s.q).to(dev)
        F = torch.empty_like(pos)
        pme.pme_reserve(plan, s.n)
        for path, name in ((pme.PME_INFLUENCE_FP32, "fp32"), (pme.PME_INFLUENCE_TENSOR, "tensor")):
            pme.pme_set_influence_path(plan, path)
            E, V = pme.pme_compute(plan, pos, q, F)
            Fh = F.cpu().numpy()
            ev = torch.zeros(7, dtype=torch.float64, device=dev)
            with torch.cuda.stream(stream):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    pme.pme_enqueue(plan, pos, q, F, ev)
                for _ in range(5):
                    g.replay()
                st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 200
                t0 = time.time()
                st.record(stream)
                for _ in range(reps):
                    g.replay()
                en.record(stream)
                torch.cuda.synchronize(dev)
                sampler.window(t0, time.time())
            pme.pme_sync(plan)
            del g
            us = 1000.0 * st.elapsed_time(en) / reps
            stages = pme.pme_profile_stages(plan, pos, q, F, reps=20)
            out[name] = {"us_per_eval": round(us, 2), "stage_us": {k: round(v, 2) for k, v in stages.items()},
                         **errs(E, V, Fh)}
        out["fp32"]["path"] = "FP32 register FFTs along k1 (int64 fixed-point charge mesh, double-float energy sums)"
        out["tensor"]["path"] = ("k1 transforms as tcgen05 matrix products, operands split into three BF16 terms, "
                                 "six term products, main and correction products in separate FP32 accumulators")
        ff = out["fp32"]
        return {"large_grid": {
            "workload": "262144 water-like atoms (87380 triplets + 2 pairs), cubic 137.9 A, 128^3, p=6, beta=0.34/A",
            "us_per_eval": ff["us_per_eval"], "stage_us": ff["stage_us"], "path": ff["path"],
            **{k: ff[k] for k in ("rel_energy_error", "rms_force_error", "rel_virial_error")},
            "tensor_core_path": out["tensor"]}}
    finally:
        pme.pme_destroy(plan)


def leg_slab(args, sampler, dist):
    """Strong scaling of one system over the ranks (only with several ranks): the 65536-atom 64^3 box divided
    into k1 slabs, one per GPU (pme_slab_*), with the two corner turns as NCCL all-to-alls and the force and
    energy sums as all-reduces through torch.distributed, all on each rank's stream. Microseconds per
    evaluation of the one system (max over ranks) and the error of the summed result against the oracle."""
    if dist.world < 2:
        return {}
    import datetime

    import torch
    import torch.distributed as tdist

    from paper_2009_12617_gb300 import pme
    from paper_2009_12617_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    g = tdist.new_group(backend="nccl", timeout=datetime.timedelta(seconds=120))
    s = wl.headline_system(seed=2)
    stream = torch.cuda.Stream(dev)
    slab = pme.pme_slab_create(s.K, s.p, s.beta, s.box, dist.world, dist.rank, stream=stream)
    try:
        lay = pme.pme_slab_layout(slab)
        B = lay["block_values"]
        pos = torch.from_numpy(s.pos).to(dev)
        q = torch.from_numpy(s.q).to(dev)
        send = torch.zeros(dist.world * B * 2, dtype=torch.float32, device=dev)
        recv, send2, recv2 = torch.zeros_like(send), torch.zeros_like(send), torch.zeros_like(send)
        F = torch.zeros_like(pos)
        ev = torch.zeros(7, dtype=torch.float64, device=dev)

        def step():
            pme.pme_slab_stage1(slab, pos, q, send)
            tdist.all_to_all_single(recv, send, group=g)
            pme.pme_slab_stage2(slab, recv, send2, ev)
            tdist.all_to_all_single(recv2, send2, group=g)
            pme.pme_slab_stage3(slab, recv2, pos, q, F)
            tdist.all_reduce(F, group=g)
            tdist.all_reduce(ev, group=g)

        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 200
        with torch.cuda.stream(stream):
            for _ in range(5):
                step()
            torch.cuda.synchronize(dev)
            dist.barrier()
            t0 = time.time()
            st.record(stream)
            for _ in range(reps):
                step()
            en.record(stream)
            torch.cuda.synchronize(dev)
            dist.barrier()
            sampler.window(t0, time.time())
        pme.pme_slab_sync(slab)
        us = dist.max(1000.0 * st.elapsed_time(en) / reps)
        out = {"slab_decomposition": {
            "workload": "one 65536-atom water-like box, 64^3, p=4, divided into k1 slabs over the ranks; corner turns "
                        "and force / energy sums by NCCL through torch.distributed",
            "ranks": dist.world, "us_per_eval": round(us, 2), "planes_rank0": list(lay["planes"]),
            "block_values": B}}
        if dist.rank == 0:
            evh = ev.cpu().numpy()
            out["slab_decomposition"]["accuracy"] = errors_vs_oracle(float(evh[0]), evh[1:], F.cpu().numpy(), s)
        return out
    finally:
        pme.pme_slab_destroy(slab)


def leg_profile(args, sampler, dist=None):
    """A short fixed sequence for ncu captures: 10 evaluations of the 65536-atom 64^3 p=4 box, then 5 of the
    262144-atom 128^3 p=6 box, then 3 more of that box with the tensor-core influence stage; eager launches on
    device arrays (six stage kernels each, in stage order)."""
    import torch

    from paper_2009_12617_gb300 import pme
    from paper_2009_12617_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    for name, s, reps in (("headline", wl.headline_system(seed=2), 10), ("large", wl.large_system(seed=3), 5),
                          ("large_tensor", wl.large_system(seed=3), 3)):
        plan = pme.pme_create(s.K, s.p, s.beta, s.box)
        try:
            if name == "large_tensor":
                pme.pme_set_influence_path(plan, pme.PME_INFLUENCE_TENSOR)
            pos = torch.from_numpy(s.pos).to(dev)
            q = torch.from_numpy(s.q).to(dev)
            F = torch.empty_like(pos)
            ev = torch.zeros(7, dtype=torch.float64, device=dev)
            pme.pme_reserve(plan, s.n)
            for _ in range(reps):
                pme.pme_enqueue(plan, pos, q, F, ev)
            pme.pme_sync(plan)
            out[name] = {"evaluations": reps, "energy": float(ev[0])}
        finally:
            pme.pme_destroy(plan)
    return {"profile": out}


def _extras():
    """Batched, served and largest-mesh legs, and the slab decomposition when there are several ranks."""
    return [leg_batched, leg_serving, leg_large, leg_slab]


if __name__ == "__main__":
    main()
