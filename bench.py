#!/usr/bin/env python
"""Throughput of the KBMOD shift-and-stack search path on a DECam-CCD-shaped stack.

One step = the whole hot path over one stack resident in HBM: psi/phi formation, the exhaustive
integer-track search with the in-line sigma-G clip and per-pixel top-K, the survivor handoff
(best n_stamps slots), 21 x 21 mean/median coadded stamps for them, the central-moment filter
of the median stamps and the de-duplication of the passing candidates.  The metric is
trajectory-epoch evaluations per second: start pixels x trajectories x epochs of the step, over
the step's device time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
  python bench.py --workload full             # 4096^2, T=100, the paper's 512 x 256 grid
  python bench.py --workload decam_refine     # off-grid refinement of the best candidates
  python bench.py --workload batch64          # 64 uneven stacks as one batch vs 64 launches

The full line runs the same step on the full-scale stack (drawn on the device with the same
recipe; numpy would take minutes).  The batch64 line times the search of 64 stacks of uneven
size and epoch count (one step = all 64) as one batch replayed from a CUDA graph, under the
schedule its autotuner picks (one persistent launch, or per-stack launches on four streams; the
tile width), against the same 64 searches as separate kb_search launches; it reports both
throughputs and the per-stack latencies (completion time from the start of the step), and
checks that both give identical results.

The decam_refine line times the refinement stage on its own: the stack is searched once, the
best --n-refine survivors are gathered, and one step = 20 Adam steps of every candidate
(bilinear sub-pixel evaluation and its gradient, kept sets fixed) plus one forward and one
backward pass at the refined tracks that also accumulates dL/dpsi and dL/dphi.

N > 1 runs one rank per GPU, each searching its own stack (stacks are independent: weak scaling,
no collective on the data path; the only all-reduce takes the slowest rank's time).  Under
torchrun the ranks are torchrun's; `python bench.py --gpus N` alone starts them itself
(torch.distributed.run on this node).  --dry-run checks that path on CPU with gloo.  --impl reference times the FP64 CPU
oracle on a bounded window of the same workload (rank 0 only).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "decam"
# workloads drawn on the device (synth.gpu_stacks.make_config_stack_torch) instead of numpy
DEVICE_DRAWN = ("full",)


class StackView:
    """The arrays of a stack (host numpy views) under make_stack's field names."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; 3 for batch64 and the reference arm; for "
                         "decam_refine, enough for ~1.5 s)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--n-stamps", type=int, default=10000)
    ap.add_argument("--n-refine", type=int, default=100000)
    ap.add_argument("--refine-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dry-run", action="store_true",
                    help="CPU-only check of the multi-rank path: ranks join a gloo group, time a "
                         "stand-in step and report as the real run does (no GPU work)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """The largest of the ranks' values of x (every rank gets it); x itself when world == 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(base, rank, stride=100):
    """Seed of rank `rank`'s own stack: ranks search independent stacks (weak scaling)."""
    return base + stride * rank


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to a scratch file (KB_CLOCKS_DIR, else the system's temporary folder);
        # the line carries their summary
        self.path = os.path.join(os.environ.get("KB_CLOCKS_DIR", tempfile.gettempdir()),
                                 "kb_bench_clocks_%d_%d.csv" % (gpu_index, os.getpid()))

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        with open(self.path) as f:
            return summarize_clock_rows(f)


def summarize_clock_rows(lines):
    """Summary of nvidia-smi rows in ClockSampler.FIELDS order (csv, no header, no units): the
    median SM clock, the largest max clock and power, and every throttle reason seen active.
    Rows without numeric clocks are skipped; a power of [N/A] counts as unknown."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm, sm_max = float(parts[1]), float(parts[2])
        except ValueError:
            continue
        try:
            power = float(parts[3])
        except ValueError:
            power = None
        rows.append((sm, sm_max, power, parts[4:]))
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for n, v in zip(names, r[3][1:]):
            if v.lower() == "active":
                reasons.add(n)
    powers = [r[2] for r in rows if r[2] is not None]
    return {"sm_mhz": statistics.median(r[0] for r in rows),
            "sm_max_mhz": max(r[1] for r in rows),
            "power_w_max": max(powers) if powers else None, "samples": len(rows),
            "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------------
# the oracle on a bounded window (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------------
_ORACLE_DATA = {}
ORACLE_MAX_SIDE = 64
# the full-scale stack's tracks reach ~2200 x 1370 pixels from a start pixel; a small window keeps
# the oracle's psi/phi of that region to a few tens of seconds
ORACLE_MAX_SIDE_OF = {"full": 8}


def _oracle_inputs(workload, stack=None):
    """The oracle's FP64 psi/phi of the workload's own stack (make_stack with the workload's
    seed: the images the GPU arm forms psi/phi from and searches), on the part of the image that
    the tracks of a centred ORACLE_MAX_SIDE^2 window of start pixels can reach, with that window
    in crop coordinates (oracle.window_inputs; generated once per process)."""
    if workload not in _ORACLE_DATA:
        import oracle
        from synth import make_stack
        if stack is None and workload in DEVICE_DRAWN:
            sys.exit("bench.py: the %s stack is drawn on the device; its CPU baseline is timed "
                     "by the GPU arm" % workload)
        s = stack if stack is not None else make_stack(workload)
        T, H, W = s.img.shape
        side = min(ORACLE_MAX_SIDE_OF.get(workload, ORACLE_MAX_SIDE), H, W)
        cx, cy = (W - side) // 2, (H - side) // 2
        psi, phi, win, _ = oracle.window_inputs(s.img, s.var, s.mask, s.psf, s.times, s.vx, s.vy,
                                                (cx, cx + side, cy, cy + side))
        _ORACLE_DATA[workload] = (psi, phi, s.times, s.vx, s.vy, win, (H, W))
    return _ORACLE_DATA[workload]


def oracle_rate(target_s, workload, stack=None):
    """Oracle search TE/s on a square window of start pixels at the centre of the workload's own
    stack (every trajectory, every epoch); the window side doubles until one run takes more than
    half of target_s (so the timed sample is about target_s/2 to 2 target_s of CPU time)."""
    import oracle
    from synth import CONFIGS
    c = CONFIGS[workload]
    psi64, phi64, times, vx, vy, win, (H, W) = _oracle_inputs(workload, stack)
    T = psi64.shape[0]
    params = dict(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"], clip=1)
    x0, y0 = win[0], win[2]
    side = 1
    while True:
        t0 = time.perf_counter()
        oracle.search(psi64, phi64, times, vx, vy, params, window=(x0, x0 + side, y0, y0 + side))
        dt = time.perf_counter() - t0
        te = side * side * len(vx) * T
        if dt * 2 > target_s or side >= win[1] - win[0]:
            break
        side *= 2
    threads = oracle.get_threads()
    return dict(value=te / dt, seconds=dt, te=te, side=side, threads=threads, T=T,
                n_traj=len(vx), H=H, W=W)


def _refine_oracle_inputs(workload, n_rand=2000):
    """Likelihood planes of the workload (FP64) and candidate tracks drawn from them without the
    CUDA path: for each injected mover the grid velocity nearest to the truth at the rounded start
    (what a grid search reports), plus random grid tracks; every epoch kept."""
    key = ("refine", workload)
    if key not in _ORACLE_DATA:
        import numpy as np
        from synth import make_likelihood_stack
        psi, phi, times, vx, vy, mv = make_likelihood_stack(workload)
        T, H, W = psi.shape
        rng = np.random.default_rng(12345)
        P = []
        for i in range(len(mv["x0"])):
            g = np.argmin((vx - mv["vx"][i]) ** 2 + (vy - mv["vy"][i]) ** 2)
            P.append([math.floor(mv["x0"][i] + 0.5), math.floor(mv["y0"][i] + 0.5), vx[g], vy[g]])
        for _ in range(n_rand):
            k = rng.integers(len(vx))
            P.append([rng.integers(0, W), rng.integers(0, H), vx[k], vy[k]])
        P = np.array(P, np.float32).astype(np.float64)
        keep = np.array([(1 << T) - 1 if T < 32 else 0xFFFFFFFF] * ((T + 31) // 32), np.uint32)
        if T % 32:
            keep[-1] = (1 << (T % 32)) - 1
        _ORACLE_DATA[key] = (psi.astype(np.float64), phi.astype(np.float64), times, P, keep)
    return _ORACLE_DATA[key]


def oracle_refine_rate(target_s, workload, n_steps):
    """Oracle refine (FP64 C Adam, one candidate per call, one thread) on the first candidates of
    _refine_oracle_inputs; the count doubles until a run takes more than half of target_s.
    Returns TE/s counting (n_steps + 1) evaluations x T epochs per candidate."""
    import oracle
    psi, phi, times, P, keep = _refine_oracle_inputs(workload)
    T = psi.shape[0]
    m = 16
    while True:
        t0 = time.perf_counter()
        for i in range(m):
            oracle.refine_adam(psi, phi, times, keep, P[i % len(P)], n_steps, 0.1, 0.2)
        dt = time.perf_counter() - t0
        if dt * 2 > target_s or m >= (1 << 20):
            break
        m *= 2
    return dict(value=m * (n_steps + 1) * T / dt, seconds=dt, n=m, T=T, threads=1)


def _device_drawn_stack(workload):
    """The GPU arm's stack of a device-drawn workload (rank 0's seed), as host arrays."""
    import torch
    from synth import CONFIGS
    from synth.gpu_stacks import make_config_stack_torch
    if not torch.cuda.is_available():
        return None
    g = make_config_stack_torch(workload, torch.device("cuda", 0), seed=CONFIGS[workload]["seed"])
    return StackView(img=g["img"].cpu().numpy(), var=g["var"].cpu().numpy(),
                     mask=g["mask"].cpu().numpy(), psf=g["psf"].cpu().numpy(), times=g["times"],
                     vx=g["vx"].cpu().numpy(), vy=g["vy"].cpu().numpy())


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload in DEVICE_DRAWN and args.workload not in _ORACLE_DATA:
        st = _device_drawn_stack(args.workload)
        if st is None:
            print(json.dumps({"impl": "reference", "unavailable": "the %s stack is drawn on the "
                              "GPU and no GPU is visible" % args.workload}))
            return
        _oracle_inputs(args.workload, st)
    if args.workload.startswith("decam_refine"):
        return run_reference_refine(args)
    if args.workload == "batch64":
        args.workload = "decam"   # the oracle on the decam planes: the same per-pair arithmetic
    r = None
    for _ in range(args.warmup):
        oracle_rate(args.cpu_seconds / 8, args.workload)
    vals = []
    t_all = 0.0
    for _ in range(args.steps):
        r = oracle_rate(args.cpu_seconds, args.workload)
        vals.append(r["value"])
        t_all += r["seconds"]
    v = statistics.median(vals)
    sample = ("oracle search (FP64 C, OpenMP) on a %dx%d start-pixel window x %d trajectories x "
              "%d epochs at the centre of the %s stack (make_stack, seed of rank 0), psi/phi "
              "formed by the oracle; TE/s" % (r["side"], r["side"], r["n_traj"], r["T"],
                                             args.workload))
    print(json.dumps({
        "impl": "reference", "metric": "trajectory-epoch evals/sec", "value": v,
        "unit": "TE/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_all / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload),
        "cpu_baseline": {"value": v, "unit": "TE/s", "cores": r["threads"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TE/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_reference_refine(args):
    for _ in range(args.warmup):
        oracle_refine_rate(args.cpu_seconds / 8, args.workload, args.refine_steps)
    vals, t_all, r = [], 0.0, None
    for _ in range(args.steps):
        r = oracle_refine_rate(args.cpu_seconds, args.workload, args.refine_steps)
        vals.append(r["value"])
        t_all += r["seconds"]
    v = statistics.median(vals)
    sample = ("oracle refine (FP64 C Adam, %d steps, one thread) of %d candidate tracks x %d "
              "epochs of the %s likelihood planes; TE/s" % (args.refine_steps, r["n"], r["T"],
                                                          args.workload))
    print(json.dumps({
        "impl": "reference", "metric": "refine trajectory-epoch evals/sec", "value": v,
        "unit": "TE/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_all / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": refine_config(args),
        "cpu_baseline": {"value": v, "unit": "TE/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TE/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def refine_config(args):
    cfg = workload_config(args.workload)
    cfg["workload"] = ("%s; refinement of the best %d survivors: %d Adam steps (lr 0.1 px, "
                       "0.2 px/day), then forward + backward with dL/dpsi, dL/dphi"
                       % (cfg["workload"], args.n_refine, args.refine_steps))
    cfg.update(n_refine=args.n_refine, refine_steps=args.refine_steps)
    return cfg


def cluster_ws_bytes(kb, n):
    import ctypes as C
    nb = C.c_size_t(0)
    kb.lib().kb_cluster_workspace_size(int(n), C.byref(nb))
    return nb.value


def search_traffic(version, workload):
    """DRAM bytes per search_kernel launch on this workload with their source, from the ncu
    summary in profiles/ (a line `traffic: <workload> <bytes> kernel_version <v> source <text>`);
    None if absent or taken on another kernel version (the counters then describe another
    kernel)."""
    import re
    p = os.path.join(ROOT, "profiles", "search_kernel_decam.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        m = re.match(r"\s*traffic:\s+(\S+)\s+([0-9.e+]+)\s+kernel_version\s+(\d+)(?:\s+source\s+(.*))?",
                     line)
        if m and m.group(1) == workload and int(m.group(3)) == version:
            return {"bytes": float(m.group(2)),
                    "source": (m.group(4) or "ncu summary in profiles/").strip()}
    return None


def workload_config(name):
    from synth import CONFIGS
    c = CONFIGS[name]
    v0, v1, ns, a0, a1, na = c["grid"]
    return {"workload": "%s: T=%d epochs of %dx%d float32, %d trajectories (%d speeds %g-%g px/day x "
                        "%d angles), K=%d, LH'>=%g, min_obs=%d, sigma-G clip 25/50/75, 2 sigma"
                        % (name, c["T"], c["H"], c["W"], ns * na, ns, v0, v1, na, c["K"],
                           c["lh_min"], c["min_obs"]),
            "T": c["T"], "H": c["H"], "W": c["W"], "n_traj": ns * na, "K": c["K"],
            "psf_k": c["psf_k"], "l2": l2_note(2 * 4 * c["T"] * c["H"] * c["W"]),
            "stack": ("%s(%r, seed=%d): the stack timed here, checked against the oracle by the "
                      "GPU tests and timed as the CPU baseline"
                      % ("synth.gpu_stacks.make_config_stack_torch" if name in DEVICE_DRAWN
                         else "synth.make_stack", name, c["seed"]))}


L2_BYTES = 126 * 2 ** 20


def l2_note(nbytes):
    """How the timed steps stand to the 126 MB L2: every bench workload's psi + phi exceed it, so
    each step reads its inputs from HBM without a flush; smaller sizes are test cases."""
    if nbytes > L2_BYTES:
        return "inputs larger than L2 (psi+phi %.2f GB)" % (nbytes / 1e9)
    return "inputs fit in L2 (psi+phi %.1f MB): a test size, not a bench workload" % (nbytes / 1e6)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2109_03296_b300 as kb
    from synth import CONFIGS, make_stack

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = CONFIGS[args.workload]
    seed = rank_seed(c["seed"], rank)
    if args.workload in DEVICE_DRAWN:
        # too large to draw with numpy in reasonable time: drawn on the device; the pinned host
        # copies feed the end-to-end leg and the CPU baseline's window
        from synth.gpu_stacks import make_config_stack_torch
        g = make_config_stack_torch(args.workload, dev, seed=seed)
        d = {k: g[k] for k in ("img", "var", "mask", "psf")}
        host = {k: v.cpu().pin_memory() for k, v in d.items()}
        s = StackView(img=host["img"].numpy(), var=host["var"].numpy(), mask=host["mask"].numpy(),
                      psf=host["psf"].numpy(), times=g["times"], vx=g["vx"].cpu().numpy(),
                      vy=g["vy"].cpu().numpy())
        vx, vy = g["vx"], g["vy"]
        del g
    else:
        s = make_stack(args.workload, seed=seed)
        # pinned host copies (for the end-to-end leg) and device-resident inputs
        host = {"img": torch.from_numpy(s.img).pin_memory(),
                "var": torch.from_numpy(s.var).pin_memory(),
                "mask": torch.from_numpy(s.mask).pin_memory(),
                "psf": torch.from_numpy(s.psf).pin_memory()}
        d = {k: v.to(dev, non_blocking=False) for k, v in host.items()}
        vx, vy = torch.from_numpy(s.vx).to(dev), torch.from_numpy(s.vy).to(dev)
    T, H, W = s.img.shape
    n_traj = len(s.vx)
    K = c["K"]
    sp = kb.SearchParams(k=K, lh_min=c["lh_min"], min_obs=c["min_obs"])
    te_step = H * W * n_traj * T
    psi = torch.empty((T, H, W), dtype=torch.float32, device=dev)
    phi = torch.empty_like(psi)
    ws = kb.alloc_workspace(kb.search_workspace_size(T, H, W, n_traj, sp), dev)
    mw = (T + 31) // 32
    out = dict(lh=torch.empty((H, W, K), dtype=torch.float32, device=dev),
               flux=torch.empty((H, W, K), dtype=torch.float32, device=dev),
               idx=torch.empty((H, W, K), dtype=torch.int32, device=dev),
               nvalid=torch.empty((H, W, K), dtype=torch.int16, device=dev),
               nkept=torch.empty((H, W, K), dtype=torch.int16, device=dev),
               mask=torch.empty((H, W, K, mw), dtype=torch.int32, device=dev))
    n_st = args.n_stamps
    cl_ws = kb.alloc_workspace(cluster_ws_bytes(kb, n_st), dev)
    stream = torch.cuda.current_stream()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a, b in kev:        # torch creates the CUDA event on first record
        a.record(stream)
        b.record(stream)

    def step(inp, kernel_events=None):
        if kernel_events is not None:
            kb.profile_events(*kernel_events)
        kb.make_psi_phi(inp["img"], inp["var"], inp["mask"], inp["psf"], psi=psi, phi=phi)
        res = kb.search(psi, phi, s.times, vx, vy, sp, workspace=ws, out=out)
        if kernel_events is not None:
            kb.profile_events(None, None)
        pix, slot, count = kb.collect(res, n_st)
        x0, y0, cvx, cvy, traj = kb.candidate_tracks(pix, slot, res, vx, vy)
        mean, med = kb.stamps(inp["img"], inp["var"], inp["mask"], s.times, x0, y0, cvx, cvy,
                              radius=10)
        moments, passed = kb.stamp_filter(med)
        keep, rep = kb.cluster(x0, y0, cvx, cvy, s.times, radius=8.0, valid=passed & (traj >= 0),
                               workspace=cl_ws)
        return dict(pix=pix, slot=slot, count=count, x0=x0, y0=y0, vx=cvx, vy=cvy, traj=traj,
                    mean=mean, median=med, moments=moments, passed=passed, keep=keep, rep=rep)

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize()
    stats = kb.search_stats(ws)
    assert stats[3] == 0, "device error flags %#x" % stats[3]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region ----
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = kb.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for i in range(args.steps):
            step(d, kernel_events=kev[i])
        e1.record(stream)
        barrier()
    kernel_ms = [a.elapsed_time(b) for a, b in kev]
    launches = kb.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world, dev)
    value = world * te_step * args.steps / (ms_max / 1e3)
    stats = kb.search_stats(ws)
    stage = kb.search_stage_counts(ws)
    pc = kb.search_pass_counts(ws)

    # ---- end to end through the C ABI from pinned host buffers ----
    # Every step copies its inputs from pinned host memory and reads its results back inside the
    # timed region.  The copy of step i+1 runs on a second stream into the other of two device
    # input buffers while step i computes (a stream of stacks in production overlaps the same
    # way); only the first copy is exposed.
    e2e = None
    if not args.no_e2e:
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        copy_stream = torch.cuda.Stream(device=dev)
        bufs = [{k: torch.empty_like(v) for k, v in d.items()} for _ in range(2)]
        ev_copied = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        ev_start = torch.cuda.Event()

        def fetch(i):
            b = i % 2
            with torch.cuda.stream(copy_stream):
                if i >= 2:
                    copy_stream.wait_event(ev_used[b])  # step i-2 is done with this buffer
                for k, v in host.items():
                    bufs[b][k].copy_(v, non_blocking=True)
                ev_copied[b].record(copy_stream)

        barrier()
        e0.record(stream)
        ev_start.record(stream)
        copy_stream.wait_event(ev_start)
        fetch(0)
        for i in range(args.steps):
            if i + 1 < args.steps:
                fetch(i + 1)
            stream.wait_event(ev_copied[i % 2])
            r = step(bufs[i % 2])
            ev_used[i % 2].record(stream)
            res_host = {k: v.to("cpu", non_blocking=True) for k, v in r.items()}
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        d2h = sum(v.numel() * v.element_size() for v in res_host.values())
        e2e_max = max_over_ranks(e2e_ms, world, dev)
        e2e = {"value": world * te_step * args.steps / (e2e_max / 1e3), "unit": "TE/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "survivors_per_step": int(res_host["count"].item())}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    peaks, peaks_src = measured_peaks()
    k_ms = statistics.median(kernel_ms)
    l2_gbs = kb.l2_read_bandwidth(device=dev)
    smem_gbs = kb.smem_read_bandwidth(device=dev)
    te_per_s_kernel = te_step / (k_ms / 1e3)
    # The search kernel's bound is its shared-memory reads: the staged bound words it sums
    # (counted per launch from its staging plan by kb_search_pass_counts) against the
    # shared-memory read bandwidth measured by kb_smem_probe in this run.
    bytes_launch = pc[0]
    achieved = bytes_launch / (k_ms / 1e3) / 1e9
    smem_all = pc[0] + pc[1] + pc[2]
    traffic = search_traffic(kb.version(), args.workload)
    line = {
        "metric": "trajectory-epoch evals/sec", "value": value, "unit": "TE/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded DECam-shaped stack)",
        "config": dict(workload_config(args.workload), n_stamps=n_st,
                       parallelism="one independent stack per GPU" if world > 1 else "1 GPU"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": smem_gbs, "unit": "GB/s",
                     "frac": achieved / smem_gbs,
                     "traffic": None if traffic is None else traffic["bytes"],
                     "traffic_source": None if traffic is None else traffic["source"],
                     "kernel": "search_kernel", "kernel_ms": k_ms,
                     "what": "on-chip: shared-memory loads of the pruning bound's staged words",
                     "peak_source": "measured in this run: kb_smem_probe, conflict-free 32-bit "
                                    "shared loads on every SM",
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "algorithmic_bytes_per_te": bytes_launch / te_step,
                     "smem_traffic": {"bound_words": pc[0], "offsets": pc[1], "tma_staged": pc[2],
                                      "direct_load_iterations": pc[3],
                                      "gbs": smem_all / (k_ms / 1e3) / 1e9,
                                      "frac": smem_all / (k_ms / 1e3) / 1e9 / smem_gbs},
                     "hbm_gather_equiv": {"bytes_per_te": 8,
                                          "achieved_gbs": te_per_s_kernel * 8 / 1e9,
                                          "hbm_peak_gbs": peaks["hbm_gbs"],
                                          "note": "8 B/TE psi+phi gather rate vs the measured HBM "
                                                  "copy peak (%s); above 1 because the bound "
                                                  "pass reuses staged tiles on chip" % peaks_src},
                     "l2_gather": {"bytes_per_te": 8, "l2_read_gbs": l2_gbs,
                                   "achieved_gbs": te_per_s_kernel * 8 / 1e9,
                                   "frac": te_per_s_kernel * 8 / 1e9 / l2_gbs,
                                   "note": "the naive gather roofline (8 B of psi+phi per "
                                           "trajectory-epoch against the L2 read bandwidth "
                                           "measured by kb_l2_probe in this run); above 1 "
                                           "because the exact bound reads its staged words from "
                                           "shared memory and only ~0.2% of pairs are gathered "
                                           "in full"}},
        "search_stats": {"te": stats[0], "full_evals": stats[1], "inserts": stats[2],
                         "full_eval_frac": stats[1] / max(1, stats[0] / T),
                         "stages": {"n_valid_ge_min_obs": stage[0], "lh_ge_lh_min": stage[1],
                                    "mean_kept_fraction": stage[2] / max(1, stage[3]),
                                    "over": "the pairs evaluated in full"}},
        "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        import oracle
        r = oracle_rate(args.cpu_seconds, args.workload, stack=s)
        n_thr = oracle.get_threads()
        oracle.set_threads(1)
        r1 = oracle_rate(args.cpu_seconds / 3, args.workload, stack=s)
        oracle.set_threads(n_thr)
        line["cpu_baseline"] = {
            "value": r["value"], "unit": "TE/s", "cores": r["threads"], "kind": "oracle",
            "sample": "FP64 C oracle search on a %dx%d start-pixel window (x %d trajectories x %d "
                      "epochs) at the centre of the timed stack, psi/phi formed by the oracle "
                      "from the same images, %.1f s" %
                      (r["side"], r["side"], r["n_traj"], r["T"], r["seconds"]),
            "single_thread": {"value": r1["value"], "unit": "TE/s",
                              "sample": "%dx%d window, one thread, %.1f s" %
                                        (r1["side"], r1["side"], r1["seconds"])}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# our arm, refinement stage
# ------------------------------------------------------------------------------------------------
def _match_movers(params, lh, movers, times, max_px=2.5):
    """Highest-L candidate whose track stays within max_px of each mover's true track at the
    first and last epoch (-1 if none)."""
    import numpy as np
    span = times[-1] - times[0]
    P = params.astype(np.float64)
    out = []
    for i in range(len(movers["x0"])):
        tx0, ty0, tvx, tvy = (movers[k][i] for k in ("x0", "y0", "vx", "vy"))
        d0 = np.hypot(P[:, 0] - tx0, P[:, 1] - ty0)
        d1 = np.hypot(P[:, 0] + P[:, 2] * span - (tx0 + tvx * span),
                      P[:, 1] + P[:, 3] * span - (ty0 + tvy * span))
        m = (d0 <= max_px) & (d1 <= max_px) & np.isfinite(lh)
        out.append(int(np.argmax(np.where(m, lh, -np.inf))) if m.any() else -1)
    return np.array(out)


def run_refine(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2109_03296_b300 as kb
    from synth import CONFIGS, make_stack

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = CONFIGS[args.workload]
    s = make_stack(args.workload, seed=rank_seed(c["seed"], rank))
    T, H, W = s.img.shape
    sp = kb.SearchParams(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"])
    rp = kb.RefineParams(n_steps=args.refine_steps)
    stream = torch.cuda.current_stream()

    # search once (not timed): the candidates and their kept sets
    dv = lambda a: torch.from_numpy(a).to(dev)
    psi, phi = kb.make_psi_phi(dv(s.img), dv(s.var), dv(s.mask), dv(s.psf))
    vx, vy = dv(s.vx), dv(s.vy)
    res = kb.search(psi, phi, s.times, vx, vy, sp)
    pix, slot, count = kb.collect(res, args.n_refine)
    params0, keep = kb.candidate_params(pix, slot, res, vx, vy)
    del res
    # the best n_refine survivors, or all of them when fewer survive
    n = min(args.n_refine, int(count.item()))
    params0, keep = params0[:n].contiguous(), keep[:n].contiguous()
    work = torch.empty_like(params0)
    gpsi = torch.empty_like(psi)
    gphi = torch.empty_like(phi)
    ones = torch.ones(n, dtype=torch.float32, device=dev)
    lh = torch.empty(n, dtype=torch.float32, device=dev)
    times = np.ascontiguousarray(s.times, np.float64)
    def stage_events(steps):
        out = {k: [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
               for k in ("refine", "fwd", "bwd")}
        for lst in out.values():
            for e in lst:       # torch creates the CUDA event on first record
                e.record(stream)
        return out

    ev = stage_events(args.steps)

    def step(p_src, i=None):
        work.copy_(p_src)
        if i is not None:
            ev["refine"][2 * i].record(stream)
        out = kb.refine(psi, phi, times, work, keep, rp, inplace=True)
        if i is not None:
            ev["refine"][2 * i + 1].record(stream)
            ev["fwd"][2 * i].record(stream)
        L, A = kb.traj_eval(psi, phi, times, work, keep)
        if i is not None:
            ev["fwd"][2 * i + 1].record(stream)
        gpsi.zero_()
        gphi.zero_()
        if i is not None:
            ev["bwd"][2 * i].record(stream)
        gp, _, _ = kb.traj_eval_backward(psi, phi, times, work, keep, ones, None, True,
                                         grad_psi=gpsi, grad_phi=gphi)
        if i is not None:
            ev["bwd"][2 * i + 1].record(stream)
        return out, L, A, gp

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.warmup):
        step(params0)
    e1.record(stream)
    torch.cuda.synchronize()
    if args.auto_steps:
        # a step takes a few ms: time enough of them to span ~1.5 s, so that the clock sampler
        # (200 ms period) sees the timed region
        per = e0.elapsed_time(e1) / max(1, args.warmup)
        args.steps = max(3, int(math.ceil(1500.0 / max(per, 1e-3))))
        args.steps = int(max_over_ranks(args.steps, world, dev))  # the same on every rank
        ev = stage_events(args.steps)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    launches0 = kb.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for i in range(args.steps):
            out = step(params0, i)
        e1.record(stream)
        barrier()
    launches = kb.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world, dev)
    evals = rp.n_steps + 1 + 2
    te_step = n * T * evals
    value = world * te_step * args.steps / (ms_max / 1e3)
    part = {k: statistics.mean(ev[k][2 * i].elapsed_time(ev[k][2 * i + 1])
                               for i in range(args.steps)) for k in ev}

    # recovery of the injected movers: grid search vs refined
    _, L1, _, L0 = out[0]
    P0, P1 = params0.cpu().numpy(), out[0][0].cpu().numpy()
    L0, L1 = L0.cpu().numpy(), L1.cpu().numpy()
    i0 = _match_movers(P0, L0, s.movers, s.times)
    i1 = _match_movers(P1, L1, s.movers, s.times)
    both = (i0 >= 0) & (i1 >= 0)
    tv = np.stack([s.movers["vx"], s.movers["vy"]], 1)
    tp = np.stack([s.movers["x0"], s.movers["y0"]], 1)
    ev0 = np.hypot(*(P0[i0[both], 2:] - tv[both]).T)
    ev1 = np.hypot(*(P1[i1[both], 2:] - tv[both]).T)
    ep0 = np.hypot(*(P0[i0[both], :2] - tp[both]).T)
    ep1 = np.hypot(*(P1[i1[both], :2] - tp[both]).T)
    gain = L1[i1[both]] / L0[i0[both]] - 1.0
    fin = np.isfinite(L0) & np.isfinite(L1)
    recovery = {
        "movers": int(len(s.movers["x0"])), "matched": int(both.sum()),
        "velocity_err_px_per_day": {"grid_median": float(np.median(ev0)),
                                    "refined_median": float(np.median(ev1)),
                                    "grid_p90": float(np.percentile(ev0, 90)),
                                    "refined_p90": float(np.percentile(ev1, 90))},
        "start_err_px": {"grid_median": float(np.median(ep0)),
                         "refined_median": float(np.median(ep1))},
        "lh_gain_median": float(np.median(gain)),
        "all_candidates": {"n": int(n), "finite": int(fin.sum()),
                           "lh_gain_median": float(np.median(L1[fin] / L0[fin] - 1.0)),
                           "frac_improved": float((L1[fin] > L0[fin]).mean())}}

    # end to end through the C ABI: candidates from pinned host memory, refined tracks and their
    # L, alpha back to the host (psi/phi stay resident; they are the search's device output)
    e2e = None
    if not args.no_e2e:
        host_p = params0.cpu().pin_memory()
        host_k = keep.cpu().pin_memory()
        h2d = host_p.numel() * 4 + host_k.numel() * 4
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            p_d = host_p.to(dev, non_blocking=True)
            k_d = host_k.to(dev, non_blocking=True)
            pr, L, A, L0_ = kb.refine(psi, phi, times, p_d, k_d, rp, inplace=True)
            Lf, Af = kb.traj_eval(psi, phi, times, pr, k_d)
            gpsi.zero_()
            gphi.zero_()
            gp, _, _ = kb.traj_eval_backward(psi, phi, times, pr, k_d, ones, None, True,
                                             grad_psi=gpsi, grad_phi=gphi)
            back = [x.to("cpu", non_blocking=True) for x in (pr, Lf, Af, gp)]
        e1.record(stream)
        barrier()
        d2h = sum(x.numel() * 4 for x in back)
        e2e_max = max_over_ranks(e0.elapsed_time(e1), world, dev)
        e2e = {"value": world * te_step * args.steps / (e2e_max / 1e3), "unit": "TE/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    r_ms = part["refine"]
    te_refine = n * T * (rp.n_steps + 1)
    # The refine kernel reads its taps through L1 (a candidate's taps stay on chip across its
    # steps; DRAM traffic is a few tens of MB): roofline = the L1/shared-memory load path (one
    # 128-byte wavefront per SM per clock), as measured in this run by kb_smem_probe, against
    # 8 float32 taps (4 of psi, 4 of phi) per trajectory-epoch.
    l1_peak = kb.smem_read_bandwidth(device=dev)
    achieved = te_refine * 32 / (r_ms / 1e3) / 1e9
    line = {
        "metric": "refine trajectory-epoch evals/sec", "value": value, "unit": "TE/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded DECam-shaped stack, "
                                                    "movers off the grid)",
        "config": dict(refine_config(args), candidates=int(n), survivors=int(count.item()),
                       parallelism="one independent stack per GPU" if world > 1 else "1 GPU",
                       l2="psi+phi %.2f GB, above L2; candidates' taps re-read every step" %
                          (2 * 4 * T * H * W / 1e9)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": l1_peak, "unit": "GB/s",
                     "frac": achieved / l1_peak, "traffic": None,
                     "kernel": "refine_kernel", "kernel_ms": r_ms,
                     "peak_source": "measured in this run: kb_smem_probe (the load path that L1 "
                                    "and shared memory share, 128 B per SM per clock)",
                     "algorithmic_bytes_per_te": 32,
                     "note": "8 x 4 B bilinear taps per trajectory-epoch, %d evaluations per "
                             "candidate; each 4 B tap occupies a 32 B sector, and the kernel is "
                             "instruction-issue bound (float-float positions, bilinear "
                             "weights, butterfly sums)" % (rp.n_steps + 1)},
        "stage_ms": part, "recovery": recovery,
        "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        r = oracle_refine_rate(args.cpu_seconds, args.workload, rp.n_steps)
        line["cpu_baseline"] = {
            "value": r["value"], "unit": "TE/s", "cores": r["threads"], "kind": "oracle",
            "sample": "FP64 C oracle Adam refine (%d steps, one candidate per call, one thread) "
                      "of %d candidate tracks x %d epochs of the workload's likelihood planes, "
                      "%.1f s" % (rp.n_steps, r["n"], r["T"], r["seconds"])}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# our arm, batched search of 64 uneven stacks
# ------------------------------------------------------------------------------------------------
def run_batch(args):
    import numpy as np
    import torch

    import paper_2109_03296_b300 as kb
    from synth.gpu_stacks import BATCH64, batch_specs, make_stack_torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    specs = batch_specs()
    stacks = []
    for (H, W, T, ns, na, nm, seed) in specs:
        st = make_stack_torch(H, W, T, ns, na, nm, rank_seed(seed, rank, 100000), dev)
        psi, phi = kb.make_psi_phi(st["img"], st["var"], st["mask"], st["psf"])
        stacks.append(dict(psi=psi, phi=phi, times=st["times"], vx=st["vx"], vy=st["vy"],
                           params=kb.SearchParams(k=8, lh_min=10.0, min_obs=min(15, T // 2))))
        del st
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    te_step = sum(s["psi"].shape[1] * s["psi"].shape[2] * s["vx"].numel() * s["psi"].shape[0]
                  for s in stacks)

    # ---- 64 separate launches (kb_search), one stream, per-stack completion events ----
    # one workspace, reused by the stream-ordered searches
    plain_out = []
    ws_need = max(kb.search_workspace_size(*s["psi"].shape, s["vx"].numel(), s["params"])
                  for s in stacks)
    plain_ws = kb.alloc_workspace(ws_need, dev)
    ev_start = torch.cuda.Event(enable_timing=True)
    ev_done = [torch.cuda.Event(enable_timing=True) for _ in stacks]

    def plain_step(record):
        outs = []
        if record:
            ev_start.record(stream)
        for i, s in enumerate(stacks):
            outs.append(kb.search(s["psi"], s["phi"], s["times"], s["vx"], s["vy"], s["params"],
                                  workspace=plain_ws,
                                  out=plain_out[i] if plain_out else None))
            if record:
                ev_done[i].record(stream)
        return outs

    plain_out.extend(plain_step(False))      # warm-up; allocates the outputs
    torch.cuda.synchronize()
    plain_ms, plain_lat = [], []
    for _ in range(max(1, args.steps)):
        plain_step(True)
        torch.cuda.synchronize()
        plain_ms.append(ev_start.elapsed_time(ev_done[-1]))
        plain_lat.append([ev_start.elapsed_time(e) for e in ev_done])

    # ---- the batch: autotuned schedule, CUDA graph replays ----
    b = kb.Batch(stacks)
    t0 = time.perf_counter()
    sched = b.autotune(reps=1)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        b.run(graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = kb.launch_count()
    batch_ms, batch_lat = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            e0.record(stream)
            b.run(graph=True)
            e1.record(stream)
            torch.cuda.synchronize()
            batch_ms.append(e0.elapsed_time(e1))
            done, tot = b.stats()
            batch_lat.append((done / 1e6).tolist())
    launches = kb.launch_count() - launches0
    pc = b.pass_counts()
    clocks = clk.summary()
    same = all(torch.equal(a[k], c[k]) for a, c in zip(plain_out, b.results)
               for k in ("idx", "nvalid", "nkept", "mask")) and \
        all(torch.equal(a[k].view(torch.int32), c[k].view(torch.int32))
            for a, c in zip(plain_out, b.results) for k in ("lh", "flux"))
    if rank != 0:
        return
    ms = statistics.median(batch_ms)
    pms = statistics.median(plain_ms)
    bl = np.array(batch_lat[-1])
    pl = np.array(plain_lat[-1])
    smem_peak = kb.smem_read_bandwidth(device=dev)
    # counted shared-memory bytes of the bound pass over all 64 stacks (kb_batch_pass_counts)
    # per step, against the shared-memory read bandwidth measured in this run
    achieved = pc[0] / (ms / 1e3) / 1e9
    sizes = {}
    for (H, W, T, ns, na, nm, seed) in specs:
        sizes["%dx%d" % (H, W)] = sizes.get("%dx%d" % (H, W), 0) + 1
    line = {
        "metric": "trajectory-epoch evals/sec", "value": world * te_step / (ms / 1e3),
        "unit": "TE/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (64 seeded DECam-recipe stacks drawn on the device)",
        "config": {"workload": "batch64: 64 stacks, sizes uniform in {512x512, 1024x2048, "
                               "2046x4094}, T uniform in 10..40, grids of 4096..32768 "
                               "trajectories (90-500 px/day, +-0.3 rad), K=8, LH'>=10, "
                               "min_obs=min(15, T/2); CUDA-graph replay of the batch, "
                               "autotuned schedule",
                   "stacks": len(stacks), "sizes": sizes, "te_per_step": te_step,
                   "l2": "inputs larger than L2 (psi+phi %.1f GB)" %
                         (sum(2 * s["psi"].numel() * 4 for s in stacks) / 1e9),
                   "parallelism": "one independent batch per GPU" if world > 1 else "1 GPU"},
        "plain": {"value": te_step / (pms / 1e3), "unit": "TE/s", "ms_per_step": pms,
                  "what": "the same 64 searches as separate kb_search launches on one stream"},
        "speedup_vs_plain": pms / ms,
        "latency_ms": {"batch": {"p50": float(np.percentile(bl, 50)),
                                 "p99": float(np.percentile(bl, 99)), "max": float(bl.max())},
                       "plain": {"p50": float(np.percentile(pl, 50)),
                                 "p99": float(np.percentile(pl, 99)), "max": float(pl.max())},
                       "definition": "completion of each stack's search from the start of the "
                                     "step (batch: device timestamps; plain: CUDA events)"},
        "schedule": {"mode": ("concurrent per-stack launches" if sched.mode == 1 else
                              "one persistent launch"),
                     "tile_order": sched.tile_order, "hot_nu2": sched.hot_nu2,
                     "score_span": sched.score_span, "stack_order": sched.stack_order,
                     "tile_cols": sched.tile_cols,
                     "tile_width": {0: "automatic per stack (64 px where the window holds >= 8 "
                                       "waves of such tiles, else 32)",
                                    1: "32 px", 2: "64 px"}[sched.tile_cols],
                     "autotune_s": tune_s},
        "results_identical_to_plain": bool(same),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                     "frac": achieved / smem_peak, "traffic": None,
                     "kernel": "search_kernel (batch) + per-stack preparation", "kernel_ms": ms,
                     "what": "on-chip: shared-memory loads of the pruning bound's staged words",
                     "peak_source": "measured in this run: kb_smem_probe, conflict-free 32-bit "
                                    "shared loads on every SM",
                     "algorithmic_bytes_per_launch": pc[0],
                     "algorithmic_bytes_per_te": pc[0] / te_step,
                     "smem_traffic": {"bound_words": pc[0], "offsets": pc[1], "tma_staged": pc[2],
                                      "direct_load_iterations": pc[3]}},
        "search_stats": tot, "clocks": clocks, "gpu_launches": launches,
        "e2e": None,
        "e2e_note": "the stacks' psi/phi are device-resident outputs of kb_make_psi_phi; the "
                    "host-to-device path is measured on the single-stack line",
    }
    if not args.no_cpu_baseline:
        r = oracle_rate(args.cpu_seconds, "decam")
        line["cpu_baseline"] = {
            "value": r["value"], "unit": "TE/s", "cores": r["threads"], "kind": "oracle",
            "sample": "FP64 C oracle search on a %dx%d start-pixel window (x %d trajectories x %d "
                      "epochs) at the centre of the decam stack, psi/phi formed by the oracle, "
                      "%.1f s" %
                      (r["side"], r["side"], r["n_traj"], r["T"], r["seconds"])}
    print(json.dumps(line), flush=True)


def launch_ranks(n, argv):
    """bench.py --gpus N run outside torchrun: start N ranks on this node (one per GPU) with
    torch.distributed.run, each running this script with the same arguments, and return their
    exit status.  Rank 0 prints the JSON line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", str(n), "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__)] + list(argv)
    return subprocess.run(cmd).returncode


def run_dry(args):
    """The multi-rank path without a GPU: every rank joins a gloo group, times a stand-in step of
    CPU work, the slowest rank's time is taken (as for the real steps) and rank 0 prints the
    line with the real workload's trajectory-epochs, one independent stack per rank."""
    import torch.distributed as dist
    from synth import CONFIGS
    rank, world, _ = dist_env()
    if world > 1:
        dist.init_process_group("gloo")
    c = CONFIGS[args.workload]
    v0, v1, ns, a0, a1, na = c["grid"]
    te_step = c["T"] * c["H"] * c["W"] * ns * na
    x = 0.0
    t0 = time.perf_counter()
    for i in range(200000 * (rank + 1)):
        x += math.sqrt(i)
    ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world, "cpu")
    seeds = [rank_seed(c["seed"], r) for r in range(world)]
    if rank == 0:
        print(json.dumps({"metric": "trajectory-epoch evals/sec", "dry_run": True,
                          "value": world * te_step * args.steps / (ms / 1e3), "unit": "TE/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms / args.steps, "scaling": "weak",
                          "config": dict(workload_config(args.workload), seeds=seeds,
                                         parallelism="one independent stack per GPU"
                                         if world > 1 else "1 GPU")}), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus:
        sys.exit("bench.py: --gpus %d but %d ranks were started" % (args.gpus, world))
    auto_steps = args.steps is None
    if auto_steps:
        # the search: the median of 5 timed steps (~0.6 s each); a batch64 step takes ~10 s and
        # a reference step ~12 s of CPU, so those time 3
        args.steps = 5 if (args.impl == "ours" and args.workload != "batch64") else 3
    refine = args.workload.startswith("decam_refine")
    args.auto_steps = auto_steps and refine and args.impl == "ours"
    if args.dry_run:
        run_dry(args)
    elif args.impl == "reference":
        run_reference(args)
    elif refine:
        run_refine(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
