"""Throughput of the LArTPC signal-simulation hot path on GB300.

One step = one whole forward pass (drift + rasterize + fluctuate + scatter-add, time-axis
FFT, wire-axis FFT x response x sum over impacts x inverse, time-axis inverse FFT; the
forward variant the autotuner keeps) over the 960-wire x 6000-tick plane with 100,000 depos
(fluctuation on).

Prints one JSON line.  `value` is depos/s of the device-resident step; `e2e` is the same
through the public API with the depos copied from pinned host memory and the waveforms
copied back inside the timed region; `error_vs_fp64` compares the bench frame with the FP64
oracle's.  Further legs: the fit step (forward + backward), Eq. 1's noise, ADC readout, the
rasterization variants, the 64-event batch and the three-plane 1,000,000-depo event.  The
headline numbers close the line (`summary`).  `--impl reference` times the FP64 CPU oracle
(the only place besides the cpu_baseline legs where this script runs it).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2104_08265_gb300 import synth  # noqa: E402

METRIC = "depos/s (full forward: drift, rasterize, fluctuate, scatter-add, 2D FFT convolution)"
L2_FLUSH_BYTES = 256 << 20          # > 126 MB of L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="wcsim", choices=["wcsim", "reference"])
    ap.add_argument("--workload", default="plane960-100k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-noise", action="store_true",
                    help="skip the forwards timed with Eq. 1's noise on, with ADC readout and "
                         "with the rasterization variants")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-event batched run (wcsim_batch_run vs 64 wcsim_run calls)")
    ap.add_argument("--no-event", action="store_true",
                    help="skip the three-plane 1,000,000-depo event")
    ap.add_argument("--soak-s", type=float, default=0.5,
                    help="untimed load before the timed loop, so the clock sampler sees the GPU busy")
    ap.add_argument("--write-traffic", nargs="+", metavar="NCU_REP",
                    help="no run: read DRAM bytes per launch from these ncu reports (ncu -i, raw "
                         "page) and write profiles/dram_traffic.json for the current sources")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_params(prm, rank):
    """Ranks are replicas: each simulates its own event of the same shape, its fluctuation
    seed offset by the rank."""
    return synth.DriftParams(**{**prm.__dict__, "seed": prm.seed + rank})


def max_over_ranks(x, ws, device):
    """The largest x over the ranks of the default process group (x itself when alone)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, steps, units_per_rank_step, max_total_ms):
    """Whole-job units per second: the units every rank processed over the slowest rank's
    time (weak scaling: fixed work per rank)."""
    return ws * steps * units_per_rank_step / (max_total_ms / 1e3)


def workload(name):
    wl = synth.make_workload(name)
    g, prm, kind, d = wl.planes[0]
    return wl, g, prm, kind, d


def config(name, g, d, prm):
    """The workload, identical in both arms of the benchmark."""
    return {"workload": name, "n_wires": g.n_wires, "n_imp": g.n_imp, "n_ticks": g.n_ticks,
            "pitch_mm": g.pitch_mm, "tick_us": g.tick_us, "n_depos": len(d),
            "fluctuate": prm.fluctuate, "l2": "flushed between timed steps (256 MB write); "
            "response + grid working set 690 MB > L2"}


# ---------------------------------------------------------------- byte / flop models
DECISION_BYTES = 64        # one binned depo decision
WEIGHT_SLOT_BYTES = 96     # its stored tick weights (24 floats)


def stage_bytes(g, n_depos, mean_bins, fused=False):
    """Algorithmic bytes per forward, by stage (summed over the launches of a stage).

    fused (the default forward): prep = the depo binning (depos read; decisions and slots
    written, read back and written in bucket order), no separate rasterization, rows_r2c =
    the binned decisions and weights read once and the time-axis spectra written, wire_pass =
    those spectra read, the response half-spectrum read and the wire-summed spectrum written.
    plain: prep = 0 (the grid is cleared inside rows_r2c as it is read), rasterize = depos in
    and 4 bytes per patch bin, rows_r2c = the grid read and its spectra written."""
    rows = g.n_rows
    nh = g.n_ticks // 2 + 1
    spec = rows * nh * 8
    out = {
        "wire_pass": spec + g.n_imp * g.n_wires * nh * 8 + g.n_wires * nh * 8,
        "rows_c2r": g.n_wires * nh * 8 + g.n_wires * g.n_ticks * 4,
    }
    if fused:
        dec = DECISION_BYTES + 4
        out.update({"prep": n_depos * (32 + dec + dec + DECISION_BYTES + WEIGHT_SLOT_BYTES),
                    "rasterize": 0,
                    "rows_r2c": n_depos * (DECISION_BYTES + WEIGHT_SLOT_BYTES) + spec})
    else:
        out.update({"prep": 0, "rasterize": n_depos * (32 + 4 * mean_bins),
                    "rows_r2c": rows * g.n_ticks * 4 + spec})
    return out


def backward_stage_bytes(g, n_depos, mean_bins, reused=False, kept2d=False):
    """Algorithmic bytes per launch of each backward stage (wcsim_run_backward with dL/dR,
    n_fw = n_wires, n_ft = n_ticks): S recomputed, S and G transformed, the wire adjoint, the
    inverse time FFT of dL/dS and the per-depo gather.  The wire adjoint reads S^ (or, kept2d,
    the forward's 2D spectra of S), G^ and H, writes dL/dR in full [n_imp][n_fw][n_ft] and
    dL/dS^, and passes G's 2D spectrum from part A to part B (written and read once).
    reused: the backward took the forward's S^ (wcsim_plane_set_reuse_forward), so S is
    neither recomputed nor transformed."""
    rows = g.n_rows
    nh = g.n_ticks // 2 + 1
    spec = rows * nh * 8                    # S^, its 2D spectrum or dL/dS^, all impacts
    wspec = g.n_wires * nh * 8              # one plane-wide half spectrum (G^, its 2D one)
    dR = g.n_imp * g.n_wires * g.n_ticks * 8
    return {
        "bwd_zero": 0,                          # the preceding wcsim_run left the grid clear
        "bwd_rasterize": 0 if reused else n_depos * (32 + 4 * mean_bins),
        "bwd_r2c_S": 0 if reused else rows * g.n_ticks * 4 + spec,
        "bwd_r2c_G": g.n_wires * g.n_ticks * 4 + wspec,
        # part A: G^ in, G's 2D spectrum out, S (or its 2D spectra) in, dL/dR out;
        # part B: G's 2D spectrum and H in, dL/dS^ out
        "bwd_wire_adjoint": (wspec + wspec + spec + dR) + (wspec + spec + spec)
                            + (wspec if kept2d else 0),   # the row kernel reads G's again
        "bwd_c2r_dS": spec + rows * g.n_ticks * 4,
        "bwd_depo_adjoint": n_depos * (32 + 20 + 4 * mean_bins),
    }


def bmin_bytes(g, n_depos):
    """Compulsory bytes of the whole step: depos in, response half-spectrum, waveforms out."""
    nh = g.n_ticks // 2 + 1
    return n_depos * 32 + g.n_imp * g.n_wires * nh * 8 + g.n_wires * g.n_ticks * 4


def fft_flops(g):
    import math
    nh = g.n_ticks // 2 + 1
    lt = math.log2(g.n_ticks)
    lw = math.log2(g.n_wires)
    fwd_rows = g.n_rows * 2.5 * g.n_ticks * lt
    wire = (g.n_imp + 1) * nh * 5 * g.n_wires * lw
    mult = g.n_imp * g.n_wires * nh * 8
    inv_rows = g.n_wires * 2.5 * g.n_ticks * lt
    return fwd_rows + wire + mult + inv_rows


STAGE_KERNEL = {"rows_r2c": "k_rows_r2c_direct", "wire_pass": "k_wire_warp",
                "rasterize": "k_rasterize", "rows_c2r": "k_rows_c2r"}
STAGE_KERNEL_FUSED = {"rows_r2c": "k_rows_r2c_fused", "wire_pass": "k_wire_warp",
                      "rows_c2r": "k_rows_c2r"}


def code_only(text):
    """C/C++ source without its comments and with runs of whitespace collapsed (string and
    character literals kept as written), so that edits to comments leave it unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_hash():
    """SHA-256 of the code (comments aside) of every CUDA source of the library."""
    import glob
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2104_08265_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(src, "*.cu")) + glob.glob(os.path.join(src, "*.cuh"))):
        h.update(code_only(open(f, encoding="utf-8").read()).encode())
    return h.hexdigest()


def kernel_base(name):
    """'void wcsim::<unnamed>::k_rows_r2c_direct<1>(wcsim::ConvDims, ...)' (ncu may shorten
    the namespace part) -> 'k_rows_r2c_direct'."""
    name = name.split("(")[0].split("::")[-1]
    return name.split("<")[0].split()[-1]


def write_traffic(reps):
    """DRAM bytes (read + write) per launch of every kernel captured in the ncu reports,
    averaged over launches, into profiles/dram_traffic.json with the hash of the sources."""
    import csv
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    acc = {}
    for rep in reps:
        out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True,
                             text=True, check=True).stdout
        rows = list(csv.reader(out.splitlines()))
        hdr, units = rows[0], rows[1]
        ki = hdr.index("Kernel Name")
        cols = [hdr.index("dram__bytes_read.sum"), hdr.index("dram__bytes_write.sum")]
        for r in rows[2:]:
            b = sum(float(r[c].replace(",", "")) * scale[units[c]] for c in cols)
            acc.setdefault(kernel_base(r[ki]), []).append(b)
    rec = {"_about": "DRAM bytes (read + write) per launch, mean over the captured launches, "
                     "from ncu --set full captures (one kernel and one launch per capture) of the "
                     "960-wire x 6000-tick plane with 100k depos; valid only while the code (comments aside) of the CUDA "
                     "sources hash to source_sha256.",
           "capture": ("CMD='python bench.py --steps 1 --warmup 1 --no-autotune --no-batch "
                       "--no-event --no-cpu-baseline --no-cufft --no-e2e --no-noise --soak-s 0'; "
                       "for K in <each kernel>; do $CMD && ncu --set full --import-source no "
                       "--clock-control none -k regex:$K -s 1 -c 1 -o prof_$K $CMD; done; then "
                       "python bench.py --write-traffic <the reports>"),
           "reports": [os.path.basename(r) for r in reps],
           "source_sha256": source_hash(),
           "bytes_per_launch": {k: float(np.mean(v)) for k, v in sorted(acc.items())}}
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec["bytes_per_launch"]))


def ncu_traffic(stage, fused=False):
    """DRAM bytes per launch of the stage's kernel from the committed ncu record, or None
    when the CUDA sources changed since the counters were taken."""
    kernels = STAGE_KERNEL_FUSED if fused else STAGE_KERNEL
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path) or stage not in kernels:
        return None
    rec = json.load(open(path))
    if source_hash() != rec.get("source_sha256"):
        return None
    return rec["bytes_per_launch"].get(kernels[stage])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, index):
        self.proc = None
        # the raw samples (summarised in the JSON line); WCSIM_CLOCKS_DIR keeps them elsewhere
        out_dir = os.environ.get("WCSIM_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, "bench_clocks_%d.csv" % os.getpid())
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_step(g, prm, R, d, threads=1):
    """Seconds of one oracle forward (rasterize on `threads` host threads, 0 = all; numpy's
    FFT for Eq. 2, one thread), and its frame."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    M = O.run(g, prm, R, d, threads=threads)
    return time.perf_counter() - t0, M


def cpu_baseline(g, prm, R, d):
    """The FP64 oracle as it stands on one full plane-frame of the workload: its rasterization
    on all host cores (bands of rows, no reduction: bit for bit the serial grid) and on one,
    numpy's single-threaded FFT for Eq. 2 in both.  Returns the record and the frame."""
    cores = host_cores()
    dt_mt, M = oracle_step(g, prm, R, d, threads=0)
    dt_1, _ = oracle_step(g, prm, R, d, threads=1)
    rec = {"value": len(d) / dt_mt, "unit": "depos/s", "cores": cores, "kind": "oracle",
           "sample": "1 full forward of the same workload (%d depos, %dx%d plane): "
                     "rasterization on %d threads, FFTs on one; %.2f s wall" %
                     (len(d), g.n_wires, g.n_ticks, cores, dt_mt),
           "single_thread": {"value": len(d) / dt_1, "unit": "depos/s", "cores": 1,
                             "wall_s": dt_1}}
    return rec, M


def frame_error(got, ref):
    """Relative L2 and max |err| / peak of a frame against the FP64 oracle's."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_over_peak": float(np.abs(got - ref).max() / np.abs(ref).max())}


REFERENCE_BUDGET_STEPS = 60     # full-workload oracle steps (one or two s each) per run, at most


def reference_sample(d, steps, warmup):
    """The depos of one reference step: the whole workload while the W + K steps stay within
    REFERENCE_BUDGET_STEPS full steps, else the first depos (whole tracks first) of a
    proportionally smaller sample (the frame and its convolution stay full size)."""
    n = len(d)
    total = max(1, steps + warmup)
    if total <= REFERENCE_BUDGET_STEPS:
        return d
    k = max(1000, n * REFERENCE_BUDGET_STEPS // total)
    return synth.Depos(p=d.p[:k], t=d.t[:k], td=d.td[:k], q=d.q[:k], id=d.id[:k])


def run_reference(args):
    """The oracle on the host cores (rank 0 only; the other ranks exit without work): W
    untimed and exactly K timed steps, each one forward of a bounded sample of the workload,
    its rasterization on every host core."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl, g, prm, kind, d = workload(args.workload)
    R = synth.make_response(g, kind)
    ds = reference_sample(d, args.steps, args.warmup)
    for _ in range(args.warmup):
        oracle_step(g, prm, R, ds, threads=0)
    times = [oracle_step(g, prm, R, ds, threads=0)[0] for _ in range(args.steps)]
    tot = sum(times)
    v = args.steps * len(ds) / tot
    cores = host_cores()
    sample = ("%d of the workload's %d depos per step (full %dx%d frame and convolution), "
              "rasterization on %d threads, FFTs on one" % (len(ds), len(d), g.n_wires,
                                                            g.n_ticks, cores))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "depos/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args.workload, g, d, prm),
            "cpu_baseline": {"value": v, "unit": "depos/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "depos/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- cuFFT comparison
def cufft_comparison(g, reps=10):
    """The same three transforms through torch.fft (cuFFT), for context only: never on
    the simulation path.  ms per transform set, averaged over `reps` after 2 warm-ups."""
    import torch
    nh = g.n_ticks // 2 + 1
    grid = torch.randn(g.n_rows, g.n_ticks, device="cuda")
    spec = torch.randn(g.n_imp, g.n_wires, nh, dtype=torch.complex64, device="cuda")
    mt = torch.randn(g.n_wires, nh, dtype=torch.complex64, device="cuda")
    ops = {"rows_r2c": lambda: torch.fft.rfft(grid, dim=1),
           "wire_fft_fwd_all_j": lambda: torch.fft.fft(spec, dim=1),
           "wire_fft_inv": lambda: torch.fft.ifft(mt, dim=0),
           "rows_c2r": lambda: torch.fft.irfft(mt, n=g.n_ticks, dim=1)}
    out = {}
    for k, f in ops.items():
        for _ in range(2):
            f()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            f()
        b.record()
        torch.cuda.synchronize()
        out[k + "_ms"] = a.elapsed_time(b) / reps
    return out


# ---------------------------------------------------------------- batched events
def batch_comparison(args, wcsim, steps=5):
    """64 independent events (planes 480/800/960 wires x 2000/6000/9600 ticks, depo counts
    log-uniform in 1e3..5e5): one wcsim_batch_run replayed from a CUDA graph vs 64 plain
    wcsim_run calls on the same planes, same stream, same GPU."""
    import torch
    wl = synth.make_workload("batch64")
    planes, depos, seqp = {}, [], []
    for e, (g, prm, kind, d) in enumerate(wl.planes):
        key = (g.n_wires, g.n_ticks, kind)
        if key not in planes:
            planes[key] = wcsim.Plane(g, prm, synth.make_response(g, kind, backend="torch"))
        seqp.append(planes[key])
        depos.append(wcsim.DeviceDepos.from_host(d))
    torch.cuda.empty_cache()
    b = wcsim.Batch(seqp, depos)
    n_depos = sum(len(d) for d in depos)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    graph.replay()
    torch.cuda.synchronize()

    def timed(fn):
        t = []
        for _ in range(steps):
            a = torch.cuda.Event(enable_timing=True); z = torch.cuda.Event(enable_timing=True)
            a.record(stream); fn(); z.record(stream)
            torch.cuda.synchronize()
            t.append(a.elapsed_time(z))
        return float(np.median(t))

    def sequential():
        for e, (pl, d, w) in enumerate(zip(seqp, depos, b.waves)):
            pl.run(d, out=w)

    sequential()
    ms_batch = timed(graph.replay)
    ms_seq = timed(sequential)
    for p in planes.values():
        p.close()
    return {"events": len(seqp), "plane_types": len(planes), "depos": n_depos,
            "batched_graph_ms": ms_batch, "sequential_ms": ms_seq,
            "speedup": ms_seq / ms_batch, "batched_depos_per_s": n_depos / (ms_batch * 1e-3),
            "note": "median of %d; the sequential arm runs each event with its plane's seed "
                    "(the batch adds the event index), same kernels otherwise" % steps}


# ---------------------------------------------------------------- full event
def event_leg(args, wcsim, flush, oracle=True):
    """The full three-plane event (800 U + 800 V + 960 W wires x 6000 ticks, 1,000,000 depos
    projected on each plane, fluctuation on): one step = the three plane forwards, device
    time with L2 flushed before each step.  Also its compulsory-byte roofline, the oracle on
    all host cores (one run: rasterization threaded, FFTs on one thread) and each plane's
    frame error against it."""
    import torch
    wl = synth.make_workload("event3p-1m")
    planes, depos, waves, Rs = [], [], [], []
    for g, prm, kind, d in wl.planes:
        R = synth.make_response(g, kind)
        Rs.append(R)
        pl = wcsim.Plane(g, prm, torch.from_numpy(R).cuda())
        dd = wcsim.DeviceDepos.from_host(d)
        if not args.no_autotune:
            pl.autotune(dd)
        planes.append(pl)
        depos.append(dd)
        waves.append(torch.empty((g.n_wires, g.n_ticks), dtype=torch.float32, device="cuda"))
    stream = torch.cuda.current_stream()

    def step():
        for pl, dd, w in zip(planes, depos, waves):
            pl.run(dd, out=w)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    te = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ts[i].record(stream)
        step()
        te[i].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(ts, te)) / args.steps
    n_event = len(wl.planes[0][3])
    bmin = sum(bmin_bytes(g, len(d)) for g, _, _, d in wl.planes)
    hbm, peak_kind = peaks()
    rec = {"planes": [g.n_wires for g, *_ in wl.planes], "n_ticks": wl.planes[0][0].n_ticks,
           "depos": n_event, "ms_per_event": ms, "depos_per_s": n_event / (ms * 1e-3),
           "plane_depos_per_s": sum(len(d) for *_, d in wl.planes) / (ms * 1e-3),
           "event_frames_per_s": 1e3 / ms,
           "step_roofline": {"bmin_bytes": bmin, "bmin_GBps": bmin / (ms * 1e-3) / 1e9,
                             "frac_of_hbm": bmin / (ms * 1e-3) / 1e9 / hbm,
                             "peak_kind": peak_kind}}
    if oracle:
        t0 = time.perf_counter()
        errs = []
        from oracle import oracle as O
        for (g, prm, kind, d), R, w in zip(wl.planes, Rs, waves):
            errs.append(frame_error(w.cpu().numpy(), O.run(g, prm, R, d, threads=0)))
        dt = time.perf_counter() - t0
        cores = host_cores()
        rec["cpu_baseline"] = {"value": n_event / dt, "unit": "depos/s", "cores": cores,
                               "kind": "oracle", "sample": "the whole event once (3 planes, "
                               "1,000,000 depos each): rasterization on %d threads, FFTs on "
                               "one; %.1f s wall" % (cores, dt)}
        rec["error_vs_fp64"] = errs
    for pl in planes:
        pl.close()
    return rec


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2104_08265_gb300 import _build, wcsim

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    _build.build()

    wl, g, prm, kind, d = workload(args.workload)
    # every rank simulates its own event: per-rank seed offset, same shapes
    prm = rank_params(prm, rank)
    R = synth.make_response(g, kind)

    cpu, M_oracle = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, M_oracle = cpu_baseline(g, prm, R, d)

    plane = wcsim.Plane(g, prm, torch.from_numpy(R).cuda())
    dd = wcsim.DeviceDepos.from_host(d)
    tune = None if args.no_autotune else plane.autotune(dd)
    fused = bool(tune and tune["forward_fused"])
    wave = torch.empty((g.n_wires, g.n_ticks), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    mean_bins = float(np.mean([(w[1] - w[0] + 1) * (w[3] - w[2] + 1)
                               for w in plane.windows(dd).cpu().numpy() if w[0] >= 0]))

    for _ in range(args.warmup):
        plane.run(dd, out=wave)
    torch.cuda.synchronize()
    # the bench frame against the FP64 oracle's (same seed, same Philox draws)
    err = frame_error(wave.cpu().numpy(), M_oracle) if M_oracle is not None else None
    if ws > 1:
        dist.barrier()

    clocks = Clocks(local)
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < args.soak_s:
        for _ in range(20):
            plane.run(dd, out=wave)
        torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        plane.run(dd, out=wave)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # per-stage breakdown, in a separate loop (the library's stage events stay out of the
    # timed steps above)
    plane.set_timing(True)
    stage_ms = {k: [] for k in wcsim.STAGES}
    for i in range(args.steps):
        flush.zero_()
        plane.run(dd, out=wave)
        torch.cuda.synchronize()
        for k, v in plane.stage_times().items():
            stage_ms[k].append(v)
    plane.set_timing(False)
    tot_ms = max_over_ranks(sum(step_ms), ws, "cuda")
    assert plane.check_flags() == 0

    def time_forward(call):
        """Mean device time of `call` (one forward) over the timed steps, L2 flushed."""
        for _ in range(args.warmup):
            call()
        ts_ = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        te_ = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ts_[i].record(stream)
            call()
            te_[i].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(ts_, te_)) / args.steps

    # ---- the same forward with Eq. 1's noise on (a low-pass amplitude spectrum): the noise
    # is added while the inverse time FFT stages its input
    noise = None
    if not args.no_noise:
        k = np.arange(g.n_ticks // 2 + 1)
        amp = (np.sqrt(g.n_ticks) / (1.0 + (k / (0.1 * g.n_ticks)) ** 2)).astype(np.float32)
        plane.set_noise(amp, seed=0x0015E)
        nms = time_forward(lambda: plane.run(dd, out=wave))
        plane.set_noise(None)
        noise = {"ms_per_step": nms, "depos_per_s": len(d) / (nms * 1e-3),
                 "model": "spectral noise per wire, A(k) = sqrt(n_t) / (1 + (k / 0.1 n_t)^2)"}

    # ---- the same forward read out as 12-bit ADC codes (wcsim_run_adc)
    adc = None
    if not args.no_noise:
        plane.set_digitizer(2.0, 2048.0, 12)
        codes = torch.empty((g.n_wires, g.n_ticks), dtype=torch.int16, device="cuda")
        ams = time_forward(lambda: plane.run_adc(dd, out=codes))
        adc = {"ms_per_step": ams, "depos_per_s": len(d) / (ams * 1e-3),
               "digitizer": "gain 2, pedestal 2048, 12 bits"}

    # ---- the rasterization variants: the exact binomial fluctuation and renormalised
    # patches, each in the same forward
    variants = {}
    if not args.no_noise:
        for name, prm_v in (("binomial_fluctuation", dataclasses.replace(prm, fluctuate=2)),
                            ("renormalized", dataclasses.replace(prm, renormalize=1))):
            plane.set_params(prm_v)
            vms = time_forward(lambda: plane.run(dd, out=wave))
            variants[name] = {"ms_per_step": vms, "depos_per_s": len(d) / (vms * 1e-3),
                              "fluctuate": prm_v.fluctuate, "renormalize": prm_v.renormalize}
        plane.set_params(prm)
        assert plane.check_flags() == 0

    # ---- forward + backward of a fit step on the same plane and depos, fluctuation off (loss
    # 1/2 |M - M_target|^2, target from D_L = 6, D_T = 10, lifetime 8 ms; the backward
    # includes dL/dR)
    fb_ms = None
    bwd_stages = None
    if not args.no_backward:
        tgt = dataclasses.replace(prm, DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0, fluctuate=0)
        plane.set_params(tgt)
        m_target = plane.run(dd).clone()
        plane.set_params(dataclasses.replace(prm, fluctuate=0))
        # the backward takes the spectra its forward just computed (same depos, mean path),
        # and dL/dR from the 2D spectra of S the forward's wire pass kept
        plane.set_reuse_forward(True, keep_wire_spectra=True)
        G = torch.empty_like(wave)
        loss = torch.empty(1, dtype=torch.float64, device="cuda")

        def fb_step():
            # G = M - M_target and the loss straight from the inverse time FFT
            plane.run_residual(dd, m_target, out=G, loss=loss)
            plane.backward(dd, G, want_resp=True)

        for _ in range(args.warmup):
            fb_step()
        torch.cuda.synchronize()
        fs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            fs[i].record(stream)
            fb_step()
            fe[i].record(stream)
        torch.cuda.synchronize()
        # the stage breakdown in a loop of its own: the library's stage events are not part
        # of the timed steps
        plane.set_timing(True)
        bwd_stage_ms = {k: [] for k in wcsim.BWD_STAGES}
        for i in range(args.steps):
            flush.zero_()
            fb_step()
            torch.cuda.synchronize()
            for k, v in plane.stage_times(backward=True).items():
                if k in bwd_stage_ms:
                    bwd_stage_ms[k].append(v)
        plane.set_timing(False)
        plane.set_reuse_forward(False)
        plane.set_params(prm)
        fb_ms = sum(s.elapsed_time(e) for s, e in zip(fs, fe)) / args.steps
        bwd_stages = {k: float(np.mean(v)) for k, v in bwd_stage_ms.items()}

    # ---- end to end through the public API with host buffers: every step uploads its depos
    # from pinned host memory and reads its frame back into pinned host memory.  As a user
    # streaming events would, the uploads, the runs and the read-backs go on three streams
    # with two sets of device buffers, so that step i's read-back and step i+1's upload
    # overlap runs; the timed region spans the first upload to the last read-back.
    e2e = None
    if not args.no_e2e:
        hp = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in
              (("p", d.p), ("t", d.t), ("td", d.td), ("q", d.q),
               ("id", d.id.view(np.int32)))}
        nbuf = 2
        dev = [{k: torch.empty_like(v, device="cuda") for k, v in hp.items()} for _ in range(nbuf)]
        dds = [wcsim.DeviceDepos(b["p"], b["t"], b["td"], b["q"], b["id"]) for b in dev]
        waves = [torch.empty((g.n_wires, g.n_ticks), dtype=torch.float32, device="cuda")
                 for _ in range(nbuf)]
        outs_h = [torch.empty((g.n_wires, g.n_ticks), dtype=torch.float32).pin_memory()
                  for _ in range(nbuf)]
        h2d = sum(v.numel() * v.element_size() for v in hp.values())
        d2h = outs_h[0].numel() * outs_h[0].element_size()
        s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
        ev = lambda: torch.cuda.Event()
        up_done = [ev() for _ in range(nbuf)]
        run_done = [ev() for _ in range(nbuf)]
        down_done = [ev() for _ in range(nbuf)]
        used = [False] * nbuf

        def e2e_steps(n):
            for i in range(n):
                b = i % nbuf
                with torch.cuda.stream(s_up):
                    if used[b]:
                        s_up.wait_event(run_done[b])          # dev[b] free again
                    for k in hp:
                        dev[b][k].copy_(hp[k], non_blocking=True)
                    up_done[b].record(s_up)
                stream.wait_event(up_done[b])
                if used[b]:
                    stream.wait_event(down_done[b])           # waves[b] read back
                plane.run(dds[b], out=waves[b], stream=stream)
                run_done[b].record(stream)
                with torch.cuda.stream(s_down):
                    s_down.wait_event(run_done[b])
                    outs_h[b].copy_(waves[b], non_blocking=True)
                    down_done[b].record(s_down)
                used[b] = True
            for b in range(nbuf):
                if used[b]:
                    stream.wait_event(down_done[b])

        e2e_steps(max(1, args.warmup))
        torch.cuda.synchronize()
        t0e = torch.cuda.Event(enable_timing=True)
        t1e = torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        s_up.wait_event(t0e)
        e2e_steps(args.steps)
        t1e.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(t0e.elapsed_time(t1e), ws, "cuda")
        e2e = {"value": job_throughput(ws, args.steps, len(d), e2e_ms), "unit": "depos/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e2e_ms / args.steps,
               "pipelining": "uploads, runs and read-backs on three streams, double-buffered",
               "l2": "not flushed: the plane's working set (690 MB) exceeds L2"}

    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_comparison(args, wcsim)

    event = None
    if rank == 0 and not args.no_event:
        event = event_leg(args, wcsim, flush, oracle=not args.no_cpu_baseline)

    cufft = None
    if rank == 0 and not args.no_cufft:
        cufft = cufft_comparison(g)
    if rank != 0:
        return
    hbm, peak_kind = peaks()
    sb = stage_bytes(g, len(d), mean_bins, fused=fused)
    bsb = backward_stage_bytes(g, len(d), mean_bins, reused=True, kept2d=True)
    avg = {k: float(np.mean(v)) for k, v in stage_ms.items()}
    stages = {k: {"ms": avg[k], "GB/s": sb[k] / (avg[k] * 1e-3) / 1e9 if avg[k] > 0 else None,
                  "alg_bytes": sb[k]} for k in avg}
    if fused:
        stages["prep"]["note"] = "depo binning (decide, count, scan, fill)"
        stages["rasterize"]["note"] = "inside rows_r2c (fused forward)"
    else:
        stages["prep"]["note"] = "no-op: the grid is cleared inside rows_r2c (consume and clear)"
    dom = max(avg, key=avg.get)
    ach = sb[dom] / (avg[dom] * 1e-3) / 1e9
    per_step = tot_ms / args.steps
    kernel = STAGE_KERNEL_FUSED.get(dom) if fused else STAGE_KERNEL.get(dom)
    launches = (6 if fused else 4) * args.steps
    step_roof = {"bmin_bytes": bmin_bytes(g, len(d)),
                 "bmin_GBps": bmin_bytes(g, len(d)) / (per_step * 1e-3) / 1e9,
                 "frac_of_hbm": bmin_bytes(g, len(d)) / (per_step * 1e-3) / 1e9 / hbm,
                 "fft_gflop": fft_flops(g) / 1e9,
                 "fft_tflops": fft_flops(g) / (per_step * 1e-3) / 1e12}
    # details first, the headline numbers last (a truncated tail of the line still shows them)
    line = {
        "metric": METRIC, "value": job_throughput(ws, args.steps, len(d), tot_ms), "unit": "depos/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config(args.workload, g, d, prm),
        "parallelism": "replicas" if ws > 1 else "1 gpu",
        "stages": stages,
        "backward_stages": ({k: {"ms": v, "alg_bytes": bsb[k],
                                 "GB/s": bsb[k] / (v * 1e-3) / 1e9 if v > 0 else None}
                             for k, v in bwd_stages.items()} if bwd_stages else None),
        "fit_step": ("wcsim_run_residual (mean path: G = M - M_target and the loss) then "
                     "wcsim_run_backward with dL/dR, the backward "
                     "taking the forward's spectra and the 2D spectra of S its wire pass kept "
                     "(wcsim_plane_set_reuse_forward mode 2)") if bwd_stages else None,
        "mean_bins_per_depo": mean_bins,
        "wall_s_timed_loop": wall,
        "cufft_comparison": cufft,
        "autotune": tune,
        "batch64": batch,
        "with_noise": noise,
        "adc_readout": adc,
        "rasterization_variants": variants or None,
        "event3p_1m": event,
        "forward_variant": "fused" if fused else "plain",
        "gpu_launches": launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
        "roofline": {"bound": "hbm", "kernel": kernel, "stage": dom, "achieved": ach,
                     "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": ncu_traffic(dom, fused), "alg_bytes": sb[dom],
                     "peak_kind": peak_kind + " (burst copy)"},
        "step_roofline": step_roof,
        "error_vs_fp64": err,
        "plane_frames_per_s": {"fwd": ws * 1e3 / per_step,
                               "fwd_bwd": (ws * 1e3 / fb_ms) if fb_ms else None},
        "fwd_bwd_ms_per_step": fb_ms,
        "summary": {"fwd_ms": per_step, "fwd_bwd_ms": fb_ms,
                    "step_frac_of_hbm": step_roof["frac_of_hbm"],
                    "dominant": [dom, ach / hbm],
                    "event3p_1m_ms": event["ms_per_event"] if event else None,
                    "batch64_speedup": batch["speedup"] if batch else None,
                    "rel_l2_vs_fp64": err["rel_l2"] if err else None},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.write_traffic:
        write_traffic(args.write_traffic)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
