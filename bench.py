"""Benchmark: MSM forward + backward (energy, forces, dE/dq, virial) throughput.

Workload (default): the 1M-atom point of the linear-scaling sweep: a periodic
cube at 0.1 atoms/A^3 with N = 1,024,000 uniform random +/-1 charges
(L = 217.15 A), B-spline order p = 4, h = 2 A, cutoff a = 8 A (M = 128,
8 levels). One step = one msm_forward (forces + virial bookkeeping) and one
msm_backward (dE/dr, dE/dq, virial) on that system, inputs resident in HBM.
L2 (129 MB) is flushed before every timed step by writing a 256 MB buffer.

Multi-GPU: replicas only -- every rank evaluates its own 1M-atom system (the
single-system path has no exchange step); value = all ranks' atoms / max time.

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on
the host cores, on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MSM fwd+bwd atoms/s at 1M atoms (FP32 vs FP64 oracle), % roofline, batch speedup"
N_HEADLINE = 1_024_000
FP32_LANES = 128          # FP32 lanes per SM (Blackwell)
FALLBACK_HBM_GBS = 6800.0  # used only when MEASURED_PEAKS.json is absent


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--atoms", type=int, default=N_HEADLINE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-atoms", type=int, default=N_HEADLINE)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the dynamic-cell and second-order timings (e.g. for a launch list of the step alone)")
    ap.add_argument("--tuning", type=int, nargs=2, metavar=("ANTERP_TZ", "SHORT_BLOCK"), default=None,
                    help="fixed launch shapes for the 1M-atom plan instead of msm_autotune")
    ap.add_argument("--level-method", choices=["auto", "ball", "spectral"], default="auto",
                    help="level stencils of the 1M-atom plan: ball kernels, the spectral method (FFTs), or "
                         "auto (msm_autotune's choice; ball with --tuning)")
    ap.add_argument("--batch-systems", type=int, default=512)
    ap.add_argument("--sweep", action="store_true",
                    help="linear-scaling sweep instead of the headline step: forward only (E, phi, F) on periodic "
                         "cubes of 1000 * 2^k atoms, k = 0 .. --sweep-kmax; prints one JSON object")
    ap.add_argument("--sweep-kmax", type=int, default=14)
    ap.add_argument("--cells", action="store_true",
                    help="cell-shape comparison instead of the headline step: forward + backward of the same number "
                         "of atoms in a periodic cube, a slab and tilted cells; prints one JSON object")
    ap.add_argument("--cells-atoms", type=int, default=128000)
    return ap.parse_args()


def workload_desc(n):
    L = (n / 0.1) ** (1 / 3)
    return ("periodic cube, %d atoms at 0.1/A^3 (L=%.2f A), uniform positions, +/-1 charges; p=4, h=2, a=8; "
            "fwd+bwd: E, F, dE/dq, virial" % (n, L))


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- roofline helpers
def stencil_flops(plan_params, info, cell, a, p):
    """Algorithmic FLOPs of one stencil phase.

    Ball levels apply the raw kernel samples s (nonzero for |h_1 o n| < 2a) to
    the omega'-prefiltered grid. s is even in x and in y, so per output the
    input rows (x0 -+ dx, y -+ dy) are first summed, (multiplicity - 1) adds
    per nonempty column of the quarter dx, dy >= 0, and each quarter sample
    then takes one FMA: points x (2 nnz_quarter + sum (mult - 1)), plus the
    prefilter, 2 x (p-1)^3 per padded point. Box levels apply the folded
    stencil: 2 x points x its nonzeros."""
    import ctypes as C

    import numpy as np

    from paper_2510_05961_gb300 import _lib
    lib = _lib.load()
    h1 = np.array(info["h1"])
    S = [int(math.ceil(2 * a / h1[d])) - 1 for d in range(3)]
    assert p == 4, "ball levels apply raw samples (and prefilter) for p = 4 only"
    g = [np.arange(-S[d], S[d] + 1) * h1[d] for d in range(3)]
    r2 = g[0][:, None, None] ** 2 + g[1][None, :, None] ** 2 + g[2][None, None, :] ** 2
    inside = r2 < (2 * a) ** 2
    quarter = inside[S[0]:, S[1]:, :]                      # dx >= 0, dy >= 0
    cols = quarter.any(axis=2)
    mult = np.ones(cols.shape)
    mult[1:, :] *= 2
    mult[:, 1:] *= 2
    per_point = 2.0 * int(np.count_nonzero(quarter)) + float(((mult - 1) * cols).sum())
    total = 0.0
    for l in range(1, info["ncomp"] + 1):
        n = info["n"][l - 1]
        pts = n[0] * n[1] * n[2]
        if info["stencil_kind"][l - 1] == 0:
            padded = (n[0] + 2 * S[0]) * (n[1] + 2 * S[1]) * (n[2] + 2 * S[2])
            total += pts * per_point + 2.0 * padded * (p - 1) ** 3
        else:
            lo = (C.c_int * 3)()
            sz = (C.c_int * 3)()
            _lib.check(lib.msm_plan_stencil(C.byref(plan_params), l, 0, None, 0, lo, sz))
            out = np.zeros(sz[0] * sz[1] * sz[2], np.float32)
            _lib.check(lib.msm_plan_stencil(C.byref(plan_params), l, 0, out.ctypes.data_as(C.c_void_p), out.size,
                                            lo, sz))
            total += 2.0 * pts * np.count_nonzero(out)
    return total


SHORT_FLOP_PER_PAIR = 40.0  # about 20 FMA per in-cutoff ordered pair (Horner gamma, gamma', E, phi, F, W)


def short_pairs(n, density, a):
    """In-cutoff ordered pairs of uniform random positions: n * density * 4/3 pi a^3."""
    return n * density * 4.0 / 3.0 * math.pi * a ** 3


def peaks(dev, clk):
    """FP32 FMA peak from the device's SM count and the maximum SM clock seen by
    nvidia-smi (else MEASURED_PEAKS.json's), HBM from MEASURED_PEAKS.json."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mp = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mp = json.load(open(path))
    mhz = (clk or {}).get("sm_max_mhz") or mp.get("sm_max_mhz") or 2070.0
    fp32 = sms * FP32_LANES * 2 * mhz * 1e6 / 1e12
    hbm = mp.get("hbm_gbs")
    return {"fp32_tflops": fp32, "sms": sms, "sm_max_mhz": mhz,
            "hbm_gbs": hbm if hbm else FALLBACK_HBM_GBS, "hbm_of": "measured" if hbm else "fallback",
            "fp32_of": "derived: %d SMs x %d lanes x 2 x %.0f MHz" % (sms, FP32_LANES, mhz)}


def level_points(info):
    return [n[0] * n[1] * n[2] for n in info["n"][:info["ncomp"]]]


def ball_sample_flops(info, a, p):
    """Algorithmic FLOPs of the level stencils in the factored form K = omega'^3 * s
    (Eq. kernel_stencil_by_conv_with_universal_coeff): per point of a ball level one
    FMA per nonzero kernel sample s (|h_1 o n| < 2a), plus the separable omega'
    prefilter, 2 (p-1) FLOP per axis per padded point. The kernel also sums the
    rows that share a column (the samples are even in x and y) before its FMAs;
    that saving is not counted as work here. Returns (flops, sample count)."""
    import numpy as np
    h1 = np.array(info["h1"])
    S = [int(math.ceil(2 * a / h1[d])) - 1 for d in range(3)]
    g = [np.arange(-S[d], S[d] + 1) * h1[d] for d in range(3)]
    nnz = int(np.count_nonzero((g[0][:, None, None] ** 2 + g[1][None, :, None] ** 2 +
                                g[2][None, None, :] ** 2) < (2 * a) ** 2))
    total = 0.0
    for n, kind in zip(info["n"][:info["ncomp"]], info["stencil_kind"]):
        if kind == 0:
            pts = n[0] * n[1] * n[2]
            padded = (n[0] + 2 * S[0]) * (n[1] + 2 * S[1]) * (n[2] + 2 * S[2])
            total += 2.0 * pts * nnz + 3 * 2.0 * (p - 1) * padded
    return total, nnz


def virial_sample_flops(info, a, p):
    """Algorithmic FLOPs of the grid virial: the autocorrelation C_d = sum_m q_m q_(m+d)
    over the unique lags of the sample ball (C_d = C_-d: half of them, the zero lag
    once), one FMA per lag per point of a ball level."""
    f, nnz = ball_sample_flops(info, a, p)
    pts = sum(n[0] * n[1] * n[2] for n, kind in zip(info["n"][:info["ncomp"]], info["stencil_kind"]) if kind == 0)
    return 2.0 * pts * (nnz + 1) / 2


def kernel_table(info, n, a, p, ph, pk, st_flops_exec, serial_note):
    """Per-phase roofline rows from serialised phase times ph (ms): algorithmic work per
    launch / time, against the binding peak (FP32 FMA or HBM)."""
    pts = level_points(info)
    f_ball, nnz = ball_sample_flops(info, a, p)
    f_vir = virial_sample_flops(info, a, p)
    rows = {}

    def add(name, kernel, bound, work, unit_work, extra=None):
        t = ph.get(name, 0.0)
        if t <= 0:
            return
        if bound == "alu":
            ach = work / (t / 1e3) / 1e12
            row = {"kernel": kernel, "bound": "alu", "ms": round(t, 4), "achieved": ach, "unit": "TFLOP/s",
                   "peak": pk["fp32_tflops"], "frac": ach / pk["fp32_tflops"], "work": work, "work_unit": unit_work}
        else:
            ach = work / (t / 1e3) / 1e9
            row = {"kernel": kernel, "bound": "hbm", "ms": round(t, 4), "achieved": ach, "unit": "GB/s",
                   "peak": pk["hbm_gbs"], "frac": ach / pk["hbm_gbs"], "work": work, "work_unit": unit_work}
        if extra:
            row.update(extra)
        rows[name] = row

    add("bin", "k_prologue, k_bin_count, k_scan_tiles, k_scan_fix, k_bin_scatter, k_bin_rank", "hbm", 36.0 * n,
        "bytes: 36 per atom (read 16, write 16 sorted + 4 permutation)")
    pairs = short_pairs(n, 0.1, a)
    add("short", "k_short", "alu", SHORT_FLOP_PER_PAIR * pairs,
        "FLOP: %.0f per in-cutoff ordered pair (about 20 FMA), %.3g pairs" % (SHORT_FLOP_PER_PAIR, pairs))
    add("anterp", "k_anterp_cols, k_anterp_sum", "alu", 2.0 * (p ** 3 + 3 * p) * n,
        "FLOP: p^3 FMA + 3p weight FMA per atom")
    add("restrict", "k_restrict (all level steps)", "hbm", 4.0 * sum(pts[l] + pts[l + 1] for l in range(len(pts) - 1)),
        "bytes: read level l, write level l+1 (4 B per point)")
    spectral = info.get("level_method", 0) == 1
    if spectral:
        fft = sum(2 * 5.0 * m * math.log2(m) + 2.0 * m + 14.0 * m for m in pts)
        add("stencil", "k_spec_z_fwd, k_spec_y (x2), k_spec_x, k_spec_z_inv", "alu", fft,
            "FLOP: forward and inverse 3-D complex FFT of every level grid at 5 N log2 N each, the product with "
            "the real spectrum (2 N) and the virial sums over |Q|^2 (14 N)",
            {"l2_bytes": 16.0 * 5 * sum(pts) - 8.0 * sum(pts), "l2_note": "five passes over the complex work "
             "buffers (read and write 8 B per point each; the first reads and the last writes 4 B real values), "
             "L2-resident at this size; the passes are bound by L2 traffic and the barriers between FFT stages, "
             "not by FP32 arithmetic"})
    else:
        add("stencil", "k_pad, k_stencil_ball, k_stencil_box", "alu", f_ball,
            "FLOP: 2 per kernel sample of the ball (%d) per point of the ball levels, plus the omega' prefilter" % nnz,
            {"executed_flops": st_flops_exec, "executed_frac": st_flops_exec / (ph["stencil"] / 1e3) / 1e12 /
             pk["fp32_tflops"] if ph.get("stencil") else None,
             "executed_note": "the kernel sums mirrored rows first (the samples are even in x and y), so it executes "
                              "fewer FLOPs than the ball count"})
    add("prolong", "k_prolong (all level steps)", "hbm", 4.0 * sum(pts[l + 1] + 2 * pts[l] for l in range(len(pts) - 1)),
        "bytes: read level l+1, read and write level l (4 B per point)")
    add("interp", "k_interp", "alu", 2.0 * 4 * p ** 3 * n, "FLOP: 4 p^3 FMA per atom (potential and gradient)")
    add("final", "k_finalize, k_energy, k_outputs", "hbm", 76.0 * n,
        "bytes: read phi (2 x 4), fields (2 x 16), q (16), permutation (4); write phi (4) and F (12) per atom")
    if spectral:
        nparts = 8 * ((n + 255) // 256) + sum(
            m[1] * -(-m[2] // min(m[2], 2048 // m[0])) for m in info["n"][:info["ncomp"]])
        add("virial", "k_virial_slices, k_virial_out (the grid sums ran in the forward's k_spec_x)", "hbm",
            48.0 * nparts, "bytes: 6 FP64 partial sums per short-range warp and per spectral x item (%d)" % nparts)
    else:
        add("virial", "k_virial_ball, k_virial_box, k_virial_slices, k_virial_out", "alu", f_vir,
            "FLOP: 2 per unique lag (half of the %d samples) per point of the ball levels (autocorrelation)" % nnz)
    add("bscale", "k_backward_scale_res", "hbm", 36.0 * n,
        "bytes: read the forward's phi and F (16) and the inverse permutation (4); write dE/dr (12) and dE/dq (4) per atom")
    return {"rows": rows, "note": serial_note}


def source_sha(src):
    p = os.path.join(ROOT, "paper_2510_05961_gb300", "csrc", src)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def read_traffic(kernel_key, src):
    """DRAM bytes per launch recorded from an ncu capture, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic_%s.txt" % kernel_key)
    if not os.path.exists(path):
        return None
    kv = {}
    for ln in open(path):
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != source_sha(src):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample(n_sample):
    """Time the FP64 oracle's forward+backward on a sample of the workload; atoms/s."""
    import numpy as np

    import oracle as O
    from paper_2510_05961_gb300 import workloads as W
    O.build()
    w = W.random_box(n_sample)
    P = O.plan_for(w)
    pos = w.pos.astype(np.float64)
    q = w.q.astype(np.float64)
    t0 = time.perf_counter()
    O.msm(P, pos, q, forces=True, virial=True)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_sample / dt, dt, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sample = 16_000  # same density, h_1 = 1.70 A and stencil radius as the 1M-atom point
    for _ in range(args.warmup):
        oracle_sample(n_sample)
    tot = 0.0
    for _ in range(args.steps):
        _, dt, cores = oracle_sample(n_sample)
        tot += dt
    ms = tot / args.steps * 1e3
    val = n_sample / (ms / 1e3)
    sample = ("oracle fwd+bwd on %d atoms of the same workload (0.1/A^3, p=4, h=2 -> h_1=1.70 A, a=8), "
              "one evaluation per step" % n_sample)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "atoms/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(N_HEADLINE), "sample_atoms": n_sample},
        "cpu_baseline": {"value": val, "unit": "atoms/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "atoms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------- batched systems
def batch_bench(dev, nsys, steps, warmup, rank=0, world=1):
    """512 independent systems (log-uniform 20-4000 atoms, open / slab / periodic):
    forward + backward of the whole batch as one captured CUDA graph, against a
    loop of single-system forward + backward calls on the same systems. With
    several ranks each evaluates its shard of the systems (no collective)."""
    import torch

    from paper_2510_05961_gb300 import Batch, Plan, shard
    from paper_2510_05961_gb300 import workloads as W

    systems = W.batch_systems(nsys=nsys)
    if world > 1:
        parts, _ = shard.shard(systems, world)
        systems = [systems[i] for i in parts[rank]]
        nsys = len(systems)
    ntot = sum(s.n for s in systems)
    batch = Batch(systems, device=dev)
    pos = torch.from_numpy(__import__("numpy").concatenate([s.pos for s in systems])).to(dev)
    q = torch.from_numpy(__import__("numpy").concatenate([s.q for s in systems])).to(dev)
    g = torch.ones(nsys, dtype=torch.float64, device=dev)
    out_f = (torch.empty(nsys, dtype=torch.float64, device=dev), None,
             torch.empty((ntot, 3), dtype=torch.float32, device=dev))
    out_b = (torch.empty((ntot, 3), dtype=torch.float32, device=dev), torch.empty(ntot, dtype=torch.float32, device=dev),
             torch.empty(9 * nsys, dtype=torch.float64, device=dev))

    def bstep():
        batch.forward(pos, q, forces=True, virial=True, phi=False, out=out_f)
        batch.backward(g, out=out_b)

    tuned = batch.autotune(pos, q)  # launch shapes for this batch, before the capture

    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            bstep()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    assert batch.status() == 0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        bstep()
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        graph.replay()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms_batch = e0.elapsed_time(e1) / steps

    plans = [Plan(s.cell, s.pbc, s.h, s.a, s.p, s.levels, max_atoms=s.n, device=dev) for s in systems]
    pos_s = [torch.from_numpy(s.pos).to(dev) for s in systems]
    q_s = [torch.from_numpy(s.q).to(dev) for s in systems]
    g1 = torch.ones(1, dtype=torch.float64, device=dev)

    def lstep():
        for pl, p_, q_ in zip(plans, pos_s, q_s):
            pl.forward(p_, q_, forces=True, virial=True, phi=False)
            pl.backward(g1)

    lstep()
    torch.cuda.synchronize(dev)
    nl = max(1, min(steps, 5))
    e0.record(st)
    for _ in range(nl):
        lstep()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms_loop = e0.elapsed_time(e1) / nl
    return {"systems": nsys, "atoms": ntot, "ms_batched_graph": ms_batch, "ms_loop_single_calls": ms_loop,
            "speedup": ms_loop / ms_batch, "atoms_per_s_batched": ntot / (ms_batch / 1e3), "tuned": tuned,
            "workload": "log-uniform 20-4000 atoms, 1/3 open, 1/3 slab (x,y periodic), 1/3 periodic, 0.08/A^3, "
                        "N(0,0.5) charges; p=4, h=2, a=8; fwd+bwd (E, F, dE/dq, virial)"}


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2510_05961_gb300 import Plan
    from paper_2510_05961_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2510_05961_gb300 import build
    build.build()

    n = args.atoms
    w = W.random_box(n, seed=3010 + rank)
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, 0, max_atoms=n, device=dev)
    pos = torch.from_numpy(w.pos).to(dev)
    q = torch.from_numpy(w.q).to(dev)
    if args.tuning:
        plan.set_tuning(*args.tuning)
    if args.level_method != "auto":
        plan.set_level_method(1 if args.level_method == "spectral" else 0)
    else:
        plan.autotune(pos, q)  # launch shapes for this workload, before the timed steps
    info = plan.info()
    g = torch.ones(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gp = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gq = torch.empty(n, dtype=torch.float32, device=dev)
    Wv = torch.empty(9, dtype=torch.float64, device=dev)
    import ctypes as C

    from paper_2510_05961_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream)
    ws = C.c_void_p(plan.workspace.data_ptr())

    def step():
        _lib.check(lib.msm_forward(plan.handle, ws, plan.workspace.numel(), n, C.c_void_p(pos.data_ptr()),
                                   C.c_void_p(q.data_ptr()), C.c_void_p(E.data_ptr()), None, C.c_void_p(F.data_ptr()),
                                   _lib.MSM_WANT_FORCES | _lib.MSM_WANT_VIRIAL, sp))
        _lib.check(lib.msm_backward(plan.handle, ws, C.c_void_p(g.data_ptr()), C.c_void_p(gp.data_ptr()),
                                    C.c_void_p(gq.data_ptr()), C.c_void_p(Wv.data_ptr()), sp))

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    assert plan.status() == 0, "device status flags set"

    plan.profile(True)
    phase_tot = {}
    launches = 0
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
        ph, nl = plan.profile_read() if i < args.steps else ({}, 0)
        for k, v in ph.items():
            phase_tot[k] = phase_tot.get(k, 0.0) + v
        launches += nl
    torch.cuda.synchronize()
    clk = clocks.stop()
    plan.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n / (ms / 1e3)

    # dynamic cell: msm_plan_set_cell, alternating a 1% larger cell and the benchmark cell, CUDA
    # events around 20 calls, under each level method
    dyn = None
    if tuple(w.pbc) == (1, 1, 1) and w.p == 4 and not args.no_extras:
        import numpy as np
        base = np.array(w.cell, np.float64)
        method0 = info["level_method"]
        dyn = {}
        for m, name in ((0, "ball"), (1, "spectral")):
            if m == 1 and not info["spectral_ok"]:
                continue
            plan.set_level_method(m)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for i in range(4):  # untimed warm-up calls
                plan.set_cell(base * (1.01 if i % 2 == 0 else 1.0))
            plan.set_cell(base)
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(20):
                plan.set_cell(base * (1.01 if i % 2 == 0 else 1.0))
            e1.record(stream)
            torch.cuda.synchronize()
            dyn["set_cell_us_" + name] = e0.elapsed_time(e1) / 20 * 1e3
        plan.set_level_method(method0)
        dyn["what"] = ("msm_plan_set_cell: new cell lengths; stencil samples, virial weights and column tables "
                       "recomputed on the device, and the spectral method's level spectra (separable sums over the "
                       "samples, on the device), whichever method the plan runs")

    # second-order backward paths (gradients through the outputs), CUDA events, 3 repetitions each:
    # force VJP (L = sum u . F: dipole grid chain, B-spline and pair Hessians) and the potential
    # gradient (one more evaluation with the upstream as charges), each after a fresh forward
    import numpy as np
    rng = np.random.default_rng(5)
    u_dev = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).to(dev)
    g_dev = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
    tv, tp = 0.0, 0.0
    for _ in range(0 if args.no_extras else 3):
        plan.forward(pos, q, forces=True, virial=False, phi=False)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        plan.force_vjp(u_dev)
        a1.record(stream)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        plan.forward(pos, g_dev, forces=True, virial=False, phi=True)
        plan.field()
        b1.record(stream)
        torch.cuda.synchronize()
        tv += a0.elapsed_time(a1) / 3
        tp += b0.elapsed_time(b1) / 3
    second = None if args.no_extras else {"force_vjp_ms": tv, "phi_grad_ms": tp,
              "what": "after a forward with forces: msm_force_vjp for a random upstream on F; the extra "
                      "evaluation with charges g plus msm_field that the upstream on phi needs"}

    # end-to-end through the public API with host buffers (copies in the timed region)
    pos_h = torch.from_numpy(w.pos).pin_memory()
    q_h = torch.from_numpy(w.q).pin_memory()
    outs = (torch.empty(1, dtype=torch.float64, pin_memory=True), torch.empty((n, 3), dtype=torch.float32,
                                                                              pin_memory=True),
            torch.empty(n, dtype=torch.float32, pin_memory=True), torch.empty((3, 3), dtype=torch.float64,
                                                                              pin_memory=True))
    for _ in range(2):
        plan.evaluate_host(pos_h, q_h, pinned_out=outs)
    e2e_steps = max(3, min(args.steps, 10))
    t_e2e = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.evaluate_host(pos_h, q_h, pinned_out=outs)
        t_e2e += time.perf_counter() - t0
    ms_e2e = t_e2e / e2e_steps * 1e3
    if world > 1:
        t = torch.tensor([ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    e2e_val = world * n / (ms_e2e / 1e3)

    # per-kernel rooflines: a serialised pass (every phase on the caller's stream, so each
    # phase's CUDA-event time is its own), 5 steps after the timed region
    pk = peaks(dev, clk)
    plan.profile(True, serial=True)
    ser = {}
    for i in range(7):
        flush.zero_()
        step()
        ph, _ = plan.profile_read()
        if i >= 2:
            for k, v in ph.items():
                ser[k] = ser.get(k, 0.0) + v / 5
    plan.profile(False)
    st_exec = stencil_flops(plan.params, info, w.cell, w.a, w.p)
    table = kernel_table(info, n, w.a, w.p, ser, pk, st_exec,
                         "phases timed one after the other on one stream (msm_profile mode 2), CUDA events, "
                         "mean of 5 steps after the timed region, L2 flushed before each step")
    # headline roofline: the dominant kernel (longest serialised phase), its algorithmic work
    # over its live phase time in the timed region (events on its own stream)
    ph_ms = {k: v / args.steps for k, v in phase_tot.items()}
    dom = max(table["rows"], key=lambda k: table["rows"][k]["ms"])
    row = table["rows"][dom]
    tms = ph_ms.get(dom, 0.0)
    if row["bound"] == "alu":
        achieved = row["work"] / (tms / 1e3) / 1e12 if tms > 0 else 0.0
        peak, unit = pk["fp32_tflops"], "TFLOP/s"
    else:
        achieved = row["work"] / (tms / 1e3) / 1e9 if tms > 0 else 0.0
        peak, unit = pk["hbm_gbs"], "GB/s"
    traffic_key = {"short": ("short_1M", "k_short.cu"), "stencil": ("stencil_ball_1M", "k_stencil.cu")}.get(dom)
    roof = {"bound": row["bound"], "kernel": row["kernel"], "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": read_traffic(*traffic_key) if traffic_key else None,
            "work": row["work"], "work_unit": row["work_unit"], "peak_note": pk["fp32_of"] if row["bound"] == "alu"
            else "HBM copy bandwidth, %s" % pk["hbm_of"],
            "live_phase_ms": {k: round(v, 4) for k, v in ph_ms.items()},
            "phase_note": "live: the short-range kernel runs on a second stream, concurrently with anterp .. "
                          "interp, so live phase times include the contention; kernels below are serialised",
            "kernels": table}

    batch_res = None
    if not args.no_batch:
        batch_res = batch_bench(dev, args.batch_systems, max(args.steps, 5), args.warmup, rank, world)
        if world > 1:
            # shards run independently; the batch's time is the slowest rank's
            t = torch.tensor([batch_res["ms_batched_graph"], float(batch_res["atoms"])], device=dev)
            tmax = t.clone()
            dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            batch_res = {"sharded": True, "ranks": world, "systems": args.batch_systems, "atoms": int(t[1].item()),
                         "ms_batched_graph_max_over_ranks": float(tmax[0].item()),
                         "atoms_per_s_batched": float(t[1].item()) / (float(tmax[0].item()) / 1e3),
                         "rank0_speedup_vs_single_calls": batch_res["speedup"], "workload": batch_res["workload"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        val, dt, cores = oracle_sample(args.cpu_sample_atoms)
        cpu = {"value": val, "unit": "atoms/s", "cores": cores, "kind": "oracle",
               "sample": "one oracle fwd+bwd (E, F, dE/dq, virial) of a %d-atom system of the same workload (same "
                         "density, p, h, a), %.1f s" % (args.cpu_sample_atoms, dt)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "atoms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(n), "atoms_per_gpu": n, "parallelism": "replicas",
                       "l2": "flushed (256 MB write) before every step", "levels": info["nlev"],
                       "M": info["M"][0],
                       "tuning": {"anterp_tz": info["anterp_tz"], "short_block": info["short_block"],
                                  "level_method": ["ball", "spectral"][info["level_method"]],
                                  "how": "fixed" if args.tuning else "msm_autotune"}},
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": e2e_val, "unit": "atoms/s", "h2d_bytes_per_step": n * 16,
                    "d2h_bytes_per_step": n * 16 + 8 + 72, "ms_per_step": ms_e2e},
            "roofline": roof, "cpu_baseline": cpu, "batch": batch_res, "dynamic_cell": dyn,
            "second_order": second,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_sweep(args):
    """Forward-only linear-scaling sweep (periodic cubes at 0.1 atoms/A^3, p=4, h=2, a=8): device time per
    forward with inputs resident and L2 flushed before every step, atoms/s, and the phase times."""
    import ctypes as C

    import torch

    from paper_2510_05961_gb300 import Plan, _lib, build
    from paper_2510_05961_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    build.build()
    lib = _lib.load()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream)
    rows = []
    for n in W.scaling_sizes(args.sweep_kmax):
        w = W.random_box(n, seed=3000 + n % 997)
        plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, 0, max_atoms=n, device=dev)
        pos = torch.from_numpy(w.pos).to(dev)
        q = torch.from_numpy(w.q).to(dev)
        plan.autotune(pos, q)  # launch shapes per size, as the main benchmark
        info = plan.info()
        E = torch.empty(1, dtype=torch.float64, device=dev)
        phi = torch.empty(n, dtype=torch.float32, device=dev)
        F = torch.empty((n, 3), dtype=torch.float32, device=dev)
        ws = C.c_void_p(plan.workspace.data_ptr())

        def fwd():
            _lib.check(lib.msm_forward(plan.handle, ws, plan.workspace.numel(), n, C.c_void_p(pos.data_ptr()),
                                       C.c_void_p(q.data_ptr()), C.c_void_p(E.data_ptr()), C.c_void_p(phi.data_ptr()),
                                       C.c_void_p(F.data_ptr()), _lib.MSM_WANT_FORCES, sp))
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            fwd()
        torch.cuda.synchronize()
        assert plan.status() == 0, "device status flags set"
        steps = max(args.steps, 5)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        plan.profile(True)
        phase = {}
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            fwd()
            evs[i][1].record(stream)
            ph, _ = plan.profile_read()
            for k, v in ph.items():
                phase[k] = phase.get(k, 0.0) + v / steps
        torch.cuda.synchronize()
        plan.profile(False)
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        peak = peaks(dev, None)["fp32_tflops"]
        spectral = info["level_method"] == 1
        fl = {"short": SHORT_FLOP_PER_PAIR * short_pairs(n, 0.1, w.a),
              "stencil": (sum(2 * 5.0 * m * math.log2(m) + 2.0 * m for m in level_points(info)) if spectral
                          else ball_sample_flops(info, w.a, w.p)[0])}
        roof = {k: (fl[k] / (phase[k] / 1e3) / 1e12 / peak if phase.get(k, 0) > 0 else None) for k in fl}
        rows.append({"atoms": n, "M": info["M"][0], "h1": round(info["h1"][0], 4), "levels": info["nlev"],
                     "tuning": [info["anterp_tz"], info["short_block"], ["ball", "spectral"][info["level_method"]]],
                     "ms_per_forward": ms, "atoms_per_s": n / (ms / 1e3),
                     "fp32_frac": roof, "phase_ms": {k: round(v, 4) for k, v in phase.items() if v > 0}})
        del plan, pos, q, E, phi, F
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": rows, "unit": "atoms/s", "workload": "periodic cubes at 0.1 atoms/A^3, uniform "
                      "positions, +/-1 charges; p=4, h=2, a=8; forward only (E, phi, F)",
                      "l2": "flushed (256 MB write) before every step", "data": "synthetic",
                      "fp32_frac_note": "algorithmic FLOP of the phase (40 per in-cutoff pair; ball method: 2 per kernel "
                                        "sample of the ball per point, plus the prefilter; spectral method: 5 N log2 N "
                                        "per forward and per inverse 3-D FFT, plus 2 N for the product) / its event "
                                        "time / the FP32 FMA peak from the SM count and "
                                        "maximum clock; the short-range phase overlaps the grid chain, so both "
                                        "include the contention"}))


def run_cells(args):
    """Forward + backward (E, F, dE/dq, virial) of N atoms at 0.1 atoms/A^3 in cells of different shape:
    periodic cube, slabs (open along z or x) and a wire (periodic along z) with lattice-summed top levels,
    and tilted periodic cells (general ball stencils, general short-range kernel). Same p = 4, a = 8 and grid counts; CUDA events, L2 flushed."""
    import numpy as np
    import torch

    from paper_2510_05961_gb300 import Plan, build
    dev = torch.device("cuda", 0)
    build.build()
    n = args.cells_atoms
    L = (n / 0.1) ** (1.0 / 3.0)
    M = 2 ** int(round(math.log2(L / 2.0)))
    shapes = {
        "cube": (np.diag([L, L, L]), (1, 1, 1)),
        "slab": (np.diag([L, L, L]), (1, 1, 0)),
        "slab_open_x": (np.diag([L, L, L]), (0, 1, 1)),
        "wire": (np.diag([L, L, L]), (0, 0, 1)),
        "sheared": (np.array([[L, 0, 0], [0.5 * L, L, 0], [0.2 * L, -0.3 * L, L]]), (1, 1, 1)),
        "hexagonal": (np.array([[L, 0, 0], [-0.5 * L, math.sqrt(3) / 2 * L, 0], [0, 0, L / (math.sqrt(3) / 2)]]),
                      (1, 1, 1)),
    }
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(77)
    frac = rng.uniform(0, 1 - 1e-6, (n, 3))  # strictly inside the cell along open axes after FP32 rounding
    q = np.concatenate([np.ones(n // 2), -np.ones(n - n // 2)]).astype(np.float32)
    rng.shuffle(q)
    rows = {}
    for name, (A, pbc) in shapes.items():
        pos = (frac @ A).astype(np.float32)
        plan = Plan(A.reshape(9), pbc, 0.0, 8.0, 4, 0, (M, M, M), max_atoms=n, device=dev)
        tp, tq = torch.from_numpy(pos).to(dev), torch.from_numpy(q).to(dev)
        plan.autotune(tp, tq)
        g = torch.ones(1, dtype=torch.float64, device=dev)
        for _ in range(max(args.warmup, 3)):
            plan.forward(tp, tq, forces=True, virial=True)
            plan.backward(g)
        torch.cuda.synchronize()
        t = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.forward(tp, tq, forces=True, virial=True)
            plan.backward(g)
            e1.record()
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1)
        ms = t / args.steps
        # per-phase CUDA-event times of one more step (outside the timed steps)
        plan.profile(True)
        flush.zero_()
        plan.forward(tp, tq, forces=True, virial=True)
        plan.backward(g)
        torch.cuda.synchronize()
        phase, _ = plan.profile_read()
        plan.profile(False)
        info = plan.info()
        rows[name] = {"ms_per_step": ms, "atoms_per_s": n / (ms / 1e3), "R": info["R"],
                      "stencil_kind": info["stencil_kind"], "pbc": list(pbc),
                      "phase_ms": {k: round(v, 4) for k, v in phase.items() if v > 0}}
        del plan
        torch.cuda.empty_cache()
    print(json.dumps({"cells": rows, "atoms": n, "M": M, "unit": "atoms/s",
                      "workload": "uniform fractional positions at 0.1 atoms/A^3, +/-1 charges; p=4, a=8, "
                                  "M=%d; fwd+bwd (E, F, dE/dq, virial)" % M}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.cells:
        run_cells(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
