"""Benchmark of the LOC ALI hot path on GB300.

Default workload: the octree cloud (64^3 root refined up to 5 levels where
the density exceeds 8x the mean, 7.9e6 leaves, 12-level rotor / 11 lines,
64 channels, 48 HEALPix directions), one step = one ALI iteration (line
parameters -> ray march -> statistical equilibrium) from LTE.  Metric:
cell-channel updates per second (one update = one (ray step, channel, line)
application of the formal solution; channels skipped by the 8-sigma window
count as updated, lines left out by --level-cutoff do not; the computed
count is reported beside it).  The same JSON line carries the serving
stream's result (--serve-requests seeded 1D models solved to 1e-4 T_ex by
the continuous-batching server: converged models/s, p50/p99 latency, and
the ratio over the plain per-model FP64-accumulation path).

Other workloads (``--workload``): ``rotor1d`` (256-shell 1D rotor cloud,
50 iterations + spectra per step), ``hotcore1d``, ``twolevel1d``,
``grid3d`` (128^3 regular grid, one iteration per step) and ``serve``
(the serving stream alone).

``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload (the only other place this script runs
the oracle is the cpu_baseline leg).

Multi-GPU: one process per GPU under torchrun; the models do not shard in
this script, so every rank solves its own replica (weak scaling, no
collective on the data path); the timing is the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import loc_inputs as LI  # noqa: E402

WINDOW = 8.0        # channel window half-width in sigma (I unchanged to FP32 beyond it)


# sources each march kernel is compiled from: a committed DRAM-traffic figure
# counts only while these files are unchanged since the capture
MARCH_SOURCES = {
    "march1d_kernel": ["k_march.cuh", "k_march1d.cu", "loc_internal.cuh"],
    "march1d_runs": ["k_march.cuh", "k_march1d.cu", "loc_internal.cuh"],
    "march3d_kernel": ["k_march.cuh", "k_march3d.cu", "walk3d.cuh", "loc_internal.cuh"],
    "march_octree_kernel": ["k_march.cuh", "k_octree.cu", "loc_internal.cuh"],
    "replay_octree_kernel": ["k_march.cuh", "k_octree.cu", "loc_internal.cuh"],
}


def sources_digest(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in MARCH_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2009_12609_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload_key):
    """DRAM bytes (read + write) per launch of `kernel` on `workload_key` from
    the committed ncu summary profiles/<kernel>_<workload>_traffic.md, scaled
    to a full launch there; None when absent or taken on other sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_key}_traffic.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        parts = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(parts) == 2 and parts[0] in ("sources_sha256", "traffic_bytes_per_launch"):
            vals[parts[0]] = parts[1].strip("`")
    if vals.get("sources_sha256") != sources_digest(kernel):
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name, n_root=128):
    if name == "rotor1d":
        mol = LI.rotor_molecule()
        model = LI.cloud1d_rotor()
        return dict(name="1D rotor cloud: 256 shells, 12 levels (11 lines), 256 channels, "
                         "50 ALI iterations + spectra",
                    key="rotor1d", mol=mol, model=model, n_iter=50, spectra=True)
    if name == "hotcore1d":
        mol = LI.rotor_molecule(n_levels=32)
        model = LI.cloud1d_rotor(t_core=150.0)
        return dict(name="1D rotor cloud with a heated centre (T_kin + 150 K exp(-(r/0.15R)^2)): "
                         "256 shells, 32 levels (31 lines), 256 channels, 50 ALI iterations + spectra",
                    key="hotcore1d", mol=mol, model=model, n_iter=50, spectra=True)
    if name == "twolevel1d":
        mol = LI.two_level_molecule()
        model = LI.cloud1d_two_level()
        return dict(name="1D two-level cloud: 32 shells, 64 channels, 20 ALI iterations + spectra",
                    key="twolevel1d", mol=mol, model=model, n_iter=20, spectra=True)
    if name == "grid3d":
        mol = LI.rotor_molecule()
        model = LI.grid3d_cloud(N=n_root)
        return dict(name=f"3D regular grid {n_root}^3, 12-level rotor (11 lines), 128 channels, "
                         "48 HEALPix directions, 1 ALI iteration",
                    key="grid3d", mol=mol, model=model, n_iter=1, spectra=False)
    if name == "octree":
        mol = LI.rotor_molecule()
        model = LI.octree_cloud(N=n_root if n_root != 128 else 64)
        n_leaf = int((model["refine"] == 0).sum())
        return dict(name=f"3D octree: {model['n_root']}^3 root refined to 5 levels where n > 8x mean "
                         f"({n_leaf} leaves), 12-level rotor (11 lines), 64 channels, "
                         "48 HEALPix directions, 1 ALI iteration",
                    key="octree", mol=mol, model=model, n_iter=1, spectra=False)
    raise SystemExit(f"unknown workload {name}")


def bytes_per_step(geometry, T, precision="fp32"):
    """Algorithmic bytes one ray step moves: its step record (1D: cell, s,
    v_los, w; octree: the 8-byte path record) and the cell's velocity /
    line width, {K, S} of every line, and the read-modify-write of the
    cell's {SIJ, ESC} per line and NORM -- plus, compensated, of their
    compensation words (FP64 accumulation: 16 bytes per line and 8 for NORM
    instead of 8 and 4)."""
    rec = {"shells1d": 16 + 4, "grid3d": 16, "octree3d": 8 + 16}[geometry]
    if precision == "fp64acc":
        return rec + 8 * T + 2 * 16 * T + 2 * 8
    acc = 2 * 8 * T + 2 * 4
    if precision == "fp32":
        acc *= 2
    return rec + 8 * T + acc


def bench_config(wl, args, world):
    """The workload's config dict, the same in both arms."""
    return {"workload": wl["name"], "iterations_per_step": wl["n_iter"],
            "channels": wl["model"]["n_ch"], "lines": len(wl["mol"]["line_nu"]),
            "window_sigmas": WINDOW, "models_per_step": world,
            "level_cutoff": args.level_cutoff,
            "parallelism": f"replicas x{world}" if world > 1 else "single"}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------
def oracle_sample(wl, budget_s=15.0):
    """Times the oracle on a bounded sample of the workload; returns
    (updates/s, cores, sample description)."""
    import oracle
    oracle.build()
    mol, model = wl["mol"], wl["model"]
    T = len(mol["line_nu"])
    nch = model["n_ch"]
    cores = oracle.n_threads()
    if model["geometry"] == "shells1d":
        segs = sum(len(oracle.paths_1d(model, j)[0]) for j in range(model["n_rays"]))
        x = oracle.lte_populations(mol, model["t_kin"])
        t0 = time.perf_counter()
        n = 0
        while True:
            x, _ = oracle.iterate_1d(mol, model, 1, x0=x)
            n += 1
            if time.perf_counter() - t0 > budget_s or n >= wl["n_iter"]:
                break
        dt = time.perf_counter() - t0
        ups = segs * nch * T * n / dt
        return ups, cores, f"{n} ALI iteration(s) of the full model ({segs} ray steps x {nch} channels x {T} lines each)"
    if model["geometry"] == "octree3d":
        # the oracle walks every lattice line of a direction: sample a small
        # octree of the same recipe (16^3 root, 3 levels), one direction
        small = LI.small_octree(N=16, levels=3, refine_frac=0.15, nside=2, n_ch=nch,
                                box_pc=0.25, abundance=1e-6, seed=5)
        small["dirs"] = small["dirs"][:1].copy()
        lm = oracle.leaf_model(small)
        x = oracle.lte_populations(mol, lm["t_kin"])
        Kp, S = oracle.line_params(mol, lm, x)
        nseg = int(sum((oracle.octree_path_sums(small, small["dirs"][0]) > 0).sum() for _ in [0]))
        t0 = time.perf_counter()
        oracle.march_octree(mol, small, Kp, S)
        dt = time.perf_counter() - t0
        # count active segments of that direction for the update rate
        N0, Lm = small["n_root"], small["levels"]
        act = 0
        for lam in range(Lm + 1):
            M = N0 << lam
            for i in range(M):
                for j in range(M):
                    if lam and i % 2 == 0 and j % 2 == 0:
                        continue
                    sg = oracle.octree_line_segments(small, small["dirs"][0], lam, i, j)
                    act += int(sg[:, 4].sum())
        ups = act * nch * T / dt
        return ups, cores, (f"ray march of one direction on a 16^3-root, 3-level octree of the same "
                            f"recipe ({act} active ray steps x {nch} channels x {T} lines)")
    # 3D: one direction, a strided subset of root rays
    N = model["n_root"]
    stride = 64
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    nseg = 0
    for r in range(0, N * N, stride):
        nseg += len(oracle.paths_grid3d(N, model["dirs"][0], r // N, r % N)[0])
    t0 = time.perf_counter()
    oracle.march_grid3d(mol, model, Kp, S, dir_range=(0, 1), ray_stride=stride)
    dt = time.perf_counter() - t0
    ups = nseg * nch * T / dt
    return ups, cores, f"ray march of direction 0, every {stride}th root ray ({nseg} ray steps x {nch} channels x {T} lines)"


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ups_list = []
    cores = 0
    sample = ""
    for i in range(args.warmup + args.steps):
        ups, cores, sample = oracle_sample(wl, budget_s=5.0)
        if i >= args.warmup:
            ups_list.append(ups)
    v = statistics.median(ups_list)
    line = {"impl": "reference", "metric": "cell-channel updates/s", "value": v,
            "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": bench_config(wl, args, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------
# replicas across ranks: every rank solves its own copy of the workload; the
# job's time is the slowest rank's, its work the sum over ranks
# ----------------------------------------------------------------------------
def max_over_ranks(x, world, device):
    """Maximum of a per-rank scalar over all ranks (all_reduce MAX on the
    process group's device: cuda under NCCL, cpu under gloo)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_throughput(units_per_rank, world, seconds_max):
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, timed by the slowest rank."""
    return units_per_rank * world / seconds_max


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def _desc_bytes(model, mol):
    b = 0
    for v in list(model.values()) + list(mol.values()):
        if isinstance(v, np.ndarray):
            b += v.nbytes
    return b


def run_gpu(args, wl):
    import torch
    import torch.distributed as dist
    from paper_2009_12609_gb300 import build, loc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    loc.load()
    peaks, peak_src = _peaks()

    mol, model = wl["mol"], wl["model"]
    T = len(mol["line_nu"])
    nch = model["n_ch"]
    is1d = model["geometry"] == "shells1d"
    R = model["radius"][-1] if is1d else None
    p_spec = np.concatenate([[0.0], (np.arange(model["n_rays"]) + 0.5) * R / model["n_rays"]]) if is1d else None
    opts = dict(max_iter=wl["n_iter"], window_sigmas=WINDOW, level_cutoff=args.level_cutoff,
                precision=args.precision)
    tune_opts = dict(window_sigmas=WINDOW, level_cutoff=args.level_cutoff, precision=args.precision)

    m = loc.Model(model, mol)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    if args.lines_per_warp or args.steps_per_chunk:
        # fixed launch shape (reproducible profiles): no autotuning
        tuned_per, tuned_chunk = args.lines_per_warp, args.steps_per_chunk
        opts.update(lines_per_pass=tuned_per, steps_per_chunk=tuned_chunk)
    else:
        tuned_per, tuned_chunk, tuned_ms = m.autotune(**tune_opts)

    def step(profile=False):
        m.reset()
        rep = m.iterate(profile=profile, **opts)
        if wl["spectra"]:
            m.spectra(0, p_spec)
        return rep

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps (outside the step events)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    reps = []
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        reps.append(step(profile=True))
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    ms_steps = [a.elapsed_time(b) for a, b in evs]
    ms_total = max_over_ranks(sum(ms_steps), world, "cuda")
    ms_step = ms_total / args.steps

    seg = reps[0]["segments"]
    iters = reps[0]["iterations"]
    # nominal updates: every channel of every (step, line) that is not left
    # out by the per-cell line truncation, counted on the device
    nominal = sum(r["nominal_updates"] for r in reps)
    upd_step = nominal / args.steps
    value = replicas_throughput(nominal, world, ms_total / 1e3)

    # dominant kernel: the ray march (CUDA events around every launch, on the
    # launching stream, inside loc_iterate)
    march_ms = sum(r["march_ms"] for r in reps)
    launches = sum(r["march_launches"] for r in reps)
    comp = sum(r["computed_updates"] for r in reps)
    se_ms = sum(r["se_ms"] for r in reps)
    par_ms = sum(r["params_ms"] for r in reps)
    per_launch_s = march_ms / 1e3 / launches
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # ALU roofline: 10 FP32-pipe operations per computed update at 128 lanes/SM
    alu_peak = n_sm * 128 * sm_max * 1e6 / 10.0 / 1e9            # Gupd/s
    achieved = comp / launches / per_launch_s / 1e9               # computed Gupd/s
    bytes_per_seg = bytes_per_step(model["geometry"], T, args.precision)
    hbm_achieved = seg * bytes_per_seg / per_launch_s / 1e9       # algorithmic GB/s
    # 1D rays cut into runs: the march is the affine + scan + run launches
    runs = is1d and tuned_chunk > 0
    replay = model["geometry"] == "octree3d" and reps[0]["path_records"] > 0
    kernel = ("march1d_runs" if runs else "march1d_kernel") if is1d else (
        ("replay_octree_kernel" if replay else "march_octree_kernel")
        if model["geometry"] == "octree3d" else "march3d_kernel")
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gupd/s",
                "frac": achieved / alu_peak,
                "traffic": committed_traffic(kernel, wl["key"]),
                "traffic_unit": "DRAM bytes per launch (ncu, cold cache)",
                "algorithmic_bytes_per_launch": seg * bytes_per_seg,
                "algorithmic_bytes_per_step": bytes_per_seg,
                "kernel": kernel,
                "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz / 10 ops per update",
                "hbm_algorithmic_gbs": hbm_achieved,
                "hbm_frac_of_measured": hbm_achieved / float(peaks["hbm_gbs"]),
                "march_ms_per_launch": per_launch_s * 1e3,
                "share_of_step": march_ms / ms_total if world == 1 else None}

    # end to end through the public API with host buffers: model creation
    # (host arrays -> device, geometry), the same solve with the tuned lines
    # per warp, populations (and spectra) back to the host
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    split = {"create_s": 0.0, "solve_s": 0.0, "readback_s": 0.0}
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        with loc.Model(model, mol) as me:
            tb = time.perf_counter()
            me.iterate(**{**opts, "lines_per_pass": tuned_per, "steps_per_chunk": tuned_chunk})
            tc = time.perf_counter()
            x = me.populations()
            d2h = x.nbytes
            if wl["spectra"]:
                sp = me.spectra(0, p_spec)
                d2h += sp.nbytes
            td = time.perf_counter()
        split["create_s"] += (tb - ta) / e2e_steps
        split["solve_s"] += (tc - tb) / e2e_steps
        split["readback_s"] += (td - tc) / e2e_steps
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, "cuda")
    e2e_val = replicas_throughput(upd_step, world, e2e_s)

    # per iteration: march (1D runs: affine, scan, run) and equilibrium; the
    # line parameters once per call (the solve prepares every later
    # iteration's); per step also the LTE reset, and for spectra line
    # parameters, step geometry and the spectrum kernel
    per_iter_launches = 4 if runs else 2
    gpu_launches = args.steps * (iters * per_iter_launches + 1 + (4 if wl["spectra"] else 1))

    m.close()
    serving = None
    if world == 1 and args.serve_requests > 0:
        serving = serve_measure(args, args.serve_requests)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            ups, cores, sample = oracle_sample(wl, budget_s=15.0)
            cpu = {"value": ups, "unit": "updates/s", "cores": cores, "kind": "oracle",
                   "sample": sample}
        line = {"metric": "cell-channel updates/s", "value": value, "unit": "updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
                "config": bench_config(wl, args, world),
                "precision": {"fp32": "FP32 march, compensated FP32 accumulation",
                              "fp32plain": "FP32 march, plain FP32 accumulation",
                              "fp64acc": "FP32 march, FP64 accumulation"}[args.precision],
                "launch": {"lines_per_warp": tuned_per, "steps_per_chunk": tuned_chunk,
                           "march_kernel": kernel},
                "work": {"ray_steps_per_iteration": seg, "octree_path_records": reps[0]["path_records"],
                         "collision_rate_table": bool(reps[0]["coll_table"]),
                         "nominal_updates_per_step": upd_step,
                         "computed_updates_per_step": comp / args.steps},
                "timing": {"l2": "flushed (256 MB write) between timed steps",
                           "clock": "CUDA events on the model's stream"},
                "computed_updates_per_s": replicas_throughput(comp, world, ms_total / 1e3),
                "models_per_s": world * 1e3 / ms_step,
                "kernel_ms_per_step": {"march": march_ms / args.steps, "se": se_ms / args.steps,
                                       "line_params": par_ms / args.steps},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": "updates/s",
                        "h2d_bytes_per_step": _desc_bytes(model, mol), "d2h_bytes_per_step": d2h,
                        "seconds_per_step": split},
                "gpu_launches": gpu_launches, "clocks": clocks,
                "wall_s_timed": wall, "peak_source": peak_src}
        if serving is not None:
            line["serving"] = serving
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def serve_measure(args, n):
    """Continuous-batching server on the stream of n seeded 1D requests:
    closed loop (all submitted at once) for the saturated converged-models/s,
    then Poisson arrivals at 0.8x that rate for p50/p99 latency; beside it the
    plain path: the first requests of the stream solved one at a time with
    FP64 per-cell accumulation, and the server on that same set."""
    import torch
    from paper_2009_12609_gb300 import build, loc
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    loc.load()
    tol, max_iter = 1e-4, 300
    cut = args.level_cutoff
    reqs = LI.serving_requests(n=n)
    mols = {L: LI.rotor_molecule(n_levels=L) for L in range(2, 21)}
    srv_opts = dict(max_slots=args.slots, mem_budget_bytes=args.mem_gb << 30,
                    iters_per_launch=4, window_sigmas=WINDOW)
    # warm-up (kernels loaded, graph captured, pool primed)
    with loc.Server(**srv_opts) as srv:
        ts = [srv.submit(r["model"], mols[r["n_levels"]], max_iter=3) for r in reqs[:8]]
        for t in ts:
            srv.poll(t, 600000)
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    with loc.Server(**srv_opts) as srv:
        t0 = time.perf_counter()
        ts = [srv.submit(r["model"], mols[r["n_levels"]], max_iter=max_iter, tol_tex=tol, level_cutoff=cut) for r in reqs]
        res = [srv.poll(t, 3600 * 1000)[0] for t in ts]
        closed_s = time.perf_counter() - t0
    clocks = clk.stop()
    conv = sum(1 for r in res if r["status"] == 0)
    upd = sum(r["updates"] for r in res)
    models_per_s = conv / closed_s          # converged models only
    # open loop: Poisson arrivals at 0.8x the saturated rate
    rate = 0.8 * models_per_s
    n_open = min(n, args.open_requests)
    arr = LI.serving_requests(n=n_open, rate_hz=rate)
    with loc.Server(**srv_opts) as srv:
        t0 = time.perf_counter()
        ts = []
        for r in arr:
            dt = r["arrival_s"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ts.append(srv.submit(r["model"], mols[r["n_levels"]], max_iter=max_iter, tol_tex=tol, level_cutoff=cut))
        lat = np.array([srv.poll(t, 3600 * 1000)[0]["latency_ms"] for t in ts])
        st = srv.stats()
    # plain per-model path with FP64 accumulation on the same requests (the
    # first n_base of the stream), and the batched server on that same set
    n_base = min(n, args.baseline_requests)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    base_conv = 0
    for r in reqs[:n_base]:
        with loc.Model(r["model"], mols[r["n_levels"]]) as m:
            rep = m.iterate(max_iter=max_iter, tol_tex=tol, precision="fp64acc", window_sigmas=WINDOW,
                            level_cutoff=cut)
            base_conv += rep["status"] == 0
    torch.cuda.synchronize()
    base_models_per_s = base_conv / (time.perf_counter() - t0)
    with loc.Server(**srv_opts) as srv:
        t0 = time.perf_counter()
        ts = [srv.submit(r["model"], mols[r["n_levels"]], max_iter=max_iter, tol_tex=tol, level_cutoff=cut)
              for r in reqs[:n_base]]
        same_conv = sum(1 for t in ts if srv.poll(t, 3600 * 1000)[0]["status"] == 0)
        same_set_models_per_s = same_conv / (time.perf_counter() - t0)
    return {"metric": "converged 1D models/s at 1e-4 T_ex", "value": models_per_s, "unit": "models/s",
            "workload": f"serving stream: {n} seeded 1D requests, shells U(32..1024), "
                        "channels {64,128,256,512}, levels U(2..20), scales x[0.1,10]",
            "requests": n, "converged": conv, "closed_loop_s": closed_s,
            "slots": args.slots, "iters_per_launch": 4, "window_sigmas": WINDOW,
            "tol_tex": tol, "max_iter": max_iter, "level_cutoff": cut,
            "updates_per_s": upd / closed_s,
            "latency_open_loop": {"rate_hz": rate, "requests": n_open,
                                  "p50_ms": float(np.percentile(lat, 50)),
                                  "p99_ms": float(np.percentile(lat, 99)),
                                  "server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"]},
            "per_model_fp64acc_models_per_s": base_models_per_s,
            "batched_same_requests_models_per_s": same_set_models_per_s,
            "same_requests": n_base,
            "speedup_vs_per_model_fp64acc": same_set_models_per_s / base_models_per_s,
            "clocks": clocks}


def run_serve(args):
    """--workload serve: the serving stream alone, as its own JSON line."""
    r = serve_measure(args, args.requests)
    line = {"metric": r["metric"], "value": r["value"], "unit": r["unit"], "n_gpus": 1,
            "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": r["workload"], "slots": r["slots"],
                       "iters_per_launch": r["iters_per_launch"], "window_sigmas": WINDOW,
                       "tol_tex": r["tol_tex"], "max_iter": r["max_iter"], "level_cutoff": r["level_cutoff"]},
            **{k: v for k, v in r.items() if k not in ("metric", "value", "unit", "workload")}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="octree",
                    choices=["rotor1d", "hotcore1d", "twolevel1d", "grid3d", "octree", "serve"])
    ap.add_argument("--requests", type=int, default=4096, help="serve: requests in the stream")
    ap.add_argument("--serve-requests", type=int, default=-1,
                    help="requests of the serving stream measured after the main workload and "
                         "reported in the same line (default: 4096 for the octree workload, "
                         "0 otherwise; 0 skips it)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32plain", "fp64acc"],
                    help="accumulation of the march: compensated FP32 (default), plain FP32, FP64")
    ap.add_argument("--open-requests", type=int, default=256, help="serve: open-loop requests")
    ap.add_argument("--baseline-requests", type=int, default=256,
                    help="serve: requests solved one at a time by the per-model FP64 path")
    ap.add_argument("--slots", type=int, default=256, help="serve: resident models")
    ap.add_argument("--mem-gb", type=int, default=64, help="serve: device memory budget")
    ap.add_argument("--n-root", type=int, default=128,
                    help="grid3d: cells per side; octree: root cells per side (default 64)")
    ap.add_argument("--lines-per-warp", type=int, default=0,
                    help="fixed lines per warp instead of the autotuned one (0: autotune)")
    ap.add_argument("--steps-per-chunk", type=int, default=0,
                    help="1D: fixed run length (-1: whole rays) instead of the autotuned one")
    ap.add_argument("--level-cutoff", type=float, default=0.0,
                    help="per-cell line truncation: skip lines whose levels hold < this fraction")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.serve_requests < 0:
        args.serve_requests = 4096 if args.workload == "octree" else 0
    if args.workload == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serve workload has no CPU arm"}))
            return
        run_serve(args)
        return
    wl = workload(args.workload, args.n_root)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
