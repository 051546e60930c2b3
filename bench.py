"""Benchmark of the EM-FEMPIC step on the drift-tube workload.

Workload: cylinder of radius 1 cm and length 10 cm on a 24 x 12 x 80 polar
Kuhn mesh (132,480 tets), order p = 2, 10^6 electrons (cold beam of radius
0.5 cm, v_z = 3e7 m/s with a 1 % spread), B0 = 1 T along the axis,
dt = 33.3 ps, FP64.  One step is one pass of the whole path: sort by tet,
gather E/B, Boris push, ray-face walk, path-integral current deposit, charge
measurement, Newmark right-hand side, device PCG solve and b update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line.  ``value`` = particle-steps per second of the whole
step (all ranks), device-timed with CUDA events, L2 flushed between steps.
With N > 1 (torchrun) each rank advances an independent replica (the
path does not shard; no collective on the data path).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec (gather+push+deposit) at p=2 and % HBM roofline; p50/p99 chunk latency"
UNIT = "particle-steps/s"
WORKLOAD = ("drift tube R=1cm L=10cm, polar Kuhn mesh 24x12x80 (132480 tets), p=2, "
            "1e6 electrons, v_z=3e7 m/s, B0=1 T, dt=33.3 ps, FP64")


def workload_name(order, n_particles, walls="beam"):
    w = WORKLOAD.replace("p=2", f"p={order}").replace("1e6 electrons", f"{n_particles:.0e} electrons"
                                                      .replace("e+0", "e"))
    return w + (", beam absorbed at z=L and re-injected at z=0" if walls == "beam" else ", reflecting walls")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, torch copy)"
    return 6800.0, "fallback 6.8 TB/s"


# ---- algorithmic bytes ---------------------------------------------------------------
def pcg_bytes_per_iteration(info):
    """Bytes one preconditioned CG iteration must move: the A arrays (8 B per
    value; at order 2 in 2x2 blocks with one 4 B column per block, else 4 B per
    entry; 4 B per value when the direction products are FP32, plus one FP64
    residual product every cg_replace_period iterations), the FP32 D, D^T, Pi
    and Pi^T arrays of the preconditioner (4 B value + 4 B column), 4 B row
    pointers, the vector passes (SpMV: p gather + q write; update: x, p, q, r
    read, x, r write; auxiliary corrections: r, t, u, dinv, dinv_L, dinv_V
    reads, t, u, z writes; direction update: p, z read, p write), and for each
    of the cheb_k - 1 Chebyshev steps of the auxiliary problems the FP32 L and
    V arrays plus five FP32 vector passes (right side, step and iterate read;
    step and iterate written).  With the Chebyshev smoother of degree ks on
    B^-1 A (cg_smooth_degree > 1): its first iterate (2x2 block inverse read,
    iterate and step written) and ks - 1 more A products (bfloat16 values,
    FP32 sums), each with the
    residual, the block inverse, the step (read and written), the iterate
    read and the next one written."""
    n1, n0 = info.n1, info.n0
    nv = 3 * info.n_nodes
    a64 = (8 * info.nnz_A + info.nnz_A) if info.order == 2 else 12 * info.nnz_A
    mats = 8 * (info.nnz_D + info.nnz_DT + 2 * info.nnz_Pi) + 4 * (3 * n1 + n0 + nv)
    aux = 8 * ((2 * n1 + 2 * n0 + n1 + n0) + (2 * nv + nv))
    k = max(1, int(info.aux_cheb_degree))
    cheb = (k - 1) * (8 * (info.nnz_L + info.nnz_V) + 4 * (n0 + nv) + 20 * (n0 + nv))
    if getattr(info, "cg_fp32_products", 0):
        # FP32 A (4 B value + a 4 B column per 2x2 block) gathering the FP32 p
        # and writing the FP32 q; update x, r from x, p, r (8 B) and q (4 B);
        # direction update reads p, z, writes p and its FP32 copy; plus, every
        # cg_replace_period iterations, one FP64 product rhs - A x
        a32 = 4 * info.nnz_A + info.nnz_A
        vec = 4 * n1 + 4 * n1 + (8 * 3 + 4 + 16) * n1 + (16 + 8 + 4) * n1
        repl = (a64 + (8 + 8 + 8 + 4) * n1) / max(1, int(info.cg_replace_period))
        ks = max(1, int(getattr(info, "cg_smooth_degree", 1)))
        a16 = 2 * info.nnz_A + info.nnz_A  # bfloat16 values, a 4 B column per 2x2 block
        smooth = 0 if ks == 1 else (16 + 8) * n1 + (ks - 1) * (a16 + (8 + 16 + 8 + 4 + 4) * n1)
        return a32 + mats + vec + aux + cheb + repl + smooth
    vec = 8 * (2 * n1 + 6 * n1 + n1 + 3 * n1)
    return a64 + mats + vec + aux + cheb


def particle_bytes_per_step(order, n_particles, occupied_tets, crossings_per_particle):
    """Bytes the particle loop must move per particle-step: the particle state
    read and written once (x, v FP64 and the tet id: 2 x (48 + 4) B) plus, per
    tet touched, its geometry (16 doubles), the gathered W1/W2 DOFs and their
    index maps, the read-modify-write of its W1 current DOFs and W0 charge
    DOFs, amortised over the particles per tet and multiplied by the tets
    visited (1 + crossings)."""
    n1, n2, n0 = {1: (6, 4, 4), 2: (20, 15, 10), 3: (45, 36, 20)}[order]
    per_tet = 128 + 8 * (n1 + n2) + 4 * (n1 + n2 + n0) + 16 * n1 + 16 * n0
    ppc = n_particles / max(1, occupied_tets)
    return 104.0 + per_tet / ppc * (1.0 + crossings_per_particle)


# ---- ranks (N > 1: one independent replica per GPU) ------------------------------------
def max_over_ranks(x, world, device=None):
    """The largest x over all ranks: the job takes as long as its slowest
    replica.  One all-reduce of a scalar, outside the timed region."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_in_rank_order(local_rank, world, build_fn, barrier_fn):
    """Compile the library once per node: local rank 0 builds, the others
    wait at the barrier and then find it up to date (two ranks compiling the
    same objects at once would overwrite each other's files)."""
    if local_rank == 0:
        build_fn()
    if world > 1:
        barrier_fn()
    if local_rank != 0:
        build_fn()


# ---- clocks -----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = [num(r[1]) for r in rows]
        smax = max(num(r[2]) for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        loaded = [s for s in sm if s == s and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(num(r[3]) for r in rows)}


# ---- oracle (CPU baseline and reference arm) ------------------------------------------
def oracle_particle_sample(cfg, n_sample, steps=1):
    """Time the oracle's particle loop (gather, push, walk, deposit, charge)
    over the first n_sample particles of the workload; returns seconds."""
    from oracle import sim as osim
    s = osim.Sim(cfg["xyz"], cfg["tets"], cfg["order"], cfg["q"], cfg["m"], cfg["weight"],
                 cfg["B0"], cfg["rho_ion"], matrices=False, bface_tag=cfg.get("bface_tag"))
    s.set_particles(cfg["x"][:n_sample], cfg["v"][:n_sample], cfg["tet"][:n_sample])
    if cfg.get("injectors"):
        s.set_injection(cfg["injectors"], cfg["inject_seed"])
    from oracle import particles as opart
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        w = s.push_walk(cfg["dt"])
        opart.measure_rho(s.topo, s.g, s.c, w["x"], w["tet"], s.qw)
        times.append(time.perf_counter() - t0)
        s.x, s.v, s.tet = w["x"], w["v"], w["tet"]
    return times


def _oracle_worker(job):
    """One worker of the multi-core oracle baseline: builds the drift-tube
    workload from its seed, steps its slice of the particles with the oracle's
    particle loop and returns the per-step times and its summed current."""
    walls, lo, hi, steps = job
    import workloads
    from oracle import particles as opart, sim as osim
    cfg = workloads.make_config(1, walls=walls)
    s = osim.Sim(cfg["xyz"], cfg["tets"], cfg["order"], cfg["q"], cfg["m"], cfg["weight"],
                 cfg["B0"], cfg["rho_ion"], matrices=False, bface_tag=cfg.get("bface_tag"))
    s.set_particles(cfg["x"][lo:hi], cfg["v"][lo:hi], cfg["tet"][lo:hi])
    if cfg.get("injectors"):
        s.set_injection(cfg["injectors"], cfg["inject_seed"])
    times, dg = [], None
    for _ in range(steps):
        t0 = time.perf_counter()
        w = s.push_walk(cfg["dt"])
        opart.measure_rho(s.topo, s.g, s.c, w["x"], w["tet"], s.qw)
        times.append(time.perf_counter() - t0)
        s.x, s.v, s.tet = w["x"], w["v"], w["tet"]
        dg = w["dg"]
    return times, dg


def oracle_particle_parallel(walls, n_sample, steps, workers=None):
    """The oracle's particle loop split by particles over the host's cores
    (spawned processes, each with its own copy of the mesh), the per-worker
    currents summed at the end.  Returns (seconds per step, workers): a step
    lasts as long as its slowest worker plus the reduction of the currents."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    bounds = np.linspace(0, n_sample, workers + 1).astype(int)
    jobs = [(walls, int(bounds[k]), int(bounds[k + 1]), steps) for k in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_oracle_worker, jobs)
    t0 = time.perf_counter()
    total = res[0][1].copy()
    for _, dg in res[1:]:
        total += dg
    t_red = time.perf_counter() - t0
    per_step = [max(r[0][k] for r in res) + t_red / steps for k in range(steps)]
    return per_step, workers


ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}


def host_cpu():
    """The host CPU's model name (x86) or Arm core part."""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key == "model name":
                return line.split(":", 1)[1].strip()
            if key == "cpu part":
                part = line.split(":", 1)[1].strip()
                return f"{ARM_PARTS.get(part, 'Arm core')} (CPU part {part})"
    except OSError:
        pass
    return None


def run_reference(args, rank, world):
    import workloads
    if rank != 0:
        return
    n_sample = args.ref_sample
    times, cores = oracle_particle_parallel(args.walls, n_sample, args.warmup + args.steps)
    timed = times[args.warmup:]
    total = sum(timed)
    value = n_sample * len(timed) / total
    sample = (f"oracle particle loop (gather, push, walk, deposit, charge) over the first "
              f"{n_sample} of the 1e6 particles per step, split by particles over {cores} host processes "
              f"({host_cpu()}), currents summed; the oracle's direct field solve is not run at this size")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(timed),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name(2, 1_000_000, args.walls), "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---- native arm -----------------------------------------------------------------------------
def run_native(args, rank, world, local_rank):
    import torch
    import workloads
    from paper_2111_12411_gb300 import Simulation

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    cfg = workloads.make_config(1, n_particles=args.particles, walls=args.walls)
    cfg["order"] = args.order
    sim = Simulation.from_config(cfg, precision=args.precision, device=local_rank,
                                 stream=stream.cuda_stream, cg_rtol=args.cg_rtol, push=args.push,
                                 cg_max_it=args.cg_max_it)
    info = sim.info
    npart = sim.n_particles
    dt = cfg["dt"]
    occupied = len(np.unique(cfg["tet"]))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        sim.step(dt)
    barrier()
    # read again after a step: the field solve's product precision is set when
    # the system is formed for this dt
    from paper_2111_12411_gb300.native import femPIC_get_info
    info = femPIC_get_info(sim.h)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    acc = {k: 0.0 for k in ("particle_ms", "field_ms", "launches", "sort_ms", "push_ms", "rhs_ms",
                            "pcg_ms", "bupdate_ms", "cg_iterations")}
    crossings = 0.0
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            sim.step(dt)
            ends[k].record(stream)
            t = sim.last_timing()
            for key in acc:
                acc[key] += t[key]
            crossings += sim.diag()["crossings"]
        barrier()
    total_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world, dev)
    K = args.steps
    value = world * npart * K / (total_ms * 1e-3)
    clocks = clk.summary()

    # ---- rooflines (dominant kernel = the CG solve; the particle kernel beside it)
    peak, peak_src = measured_peaks()
    iters = acc["cg_iterations"] / K
    pcg_bytes = pcg_bytes_per_iteration(info) * (iters + 1.0)
    pcg_ms = acc["pcg_ms"] / K
    pcg_gbs = pcg_bytes / (pcg_ms * 1e-3) / 1e9
    cross_pp = crossings / (K * max(1, npart))
    pbytes = particle_bytes_per_step(info.order, npart, occupied, cross_pp) * npart
    push_ms = acc["push_ms"] / K
    push_gbs = pbytes / (push_ms * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            per_it = json.load(open(prof)).get("k_pcg_bytes_per_iteration")
            # counters taken on an earlier build of k_pcg are not carried over
            tj = json.load(open(prof))
            if (tj.get("aux_cheb_degree", 1) != info.aux_cheb_degree
                    or tj.get("cg_fp32_products", 0) != getattr(info, "cg_fp32_products", 0)
                    or tj.get("cg_smooth_degree", 1) != getattr(info, "cg_smooth_degree", 1)):
                per_it = None
            traffic = per_it * (iters + 1.0) if per_it else None
        except (OSError, ValueError):
            traffic = None
    dominant_is_pcg = acc["pcg_ms"] >= acc["push_ms"]
    roof_pcg = {"kernel": "k_pcg (device PCG, one cooperative launch per step)", "bound": "hbm",
                "achieved": pcg_gbs, "peak": peak, "unit": "GB/s", "frac": pcg_gbs / peak,
                "traffic": traffic, "peak_source": peak_src + " of measured" if "measured" in peak_src else peak_src,
                "bytes_per_launch": pcg_bytes, "cg_iterations_per_launch": iters,
                "ms_per_launch": pcg_ms}
    part_traffic = None
    if os.path.exists(prof) and info.order == 2 and npart == 1_000_000 and args.precision == "fp64" \
            and args.walls == "beam" and args.push == "boris":
        try:
            part_traffic = json.load(open(prof)).get("k_particle_fast_dram_bytes_per_launch")
        except (OSError, ValueError):
            part_traffic = None
    roof_part = {"kernel": "k_particle (gather, push, walk, deposit, charge)", "bound": "hbm",
                 "achieved": push_gbs, "peak": peak, "unit": "GB/s", "frac": push_gbs / peak,
                 "traffic": part_traffic, "bytes_per_launch": pbytes, "ms_per_launch": push_ms,
                 "crossings_per_particle": cross_pp, "particles_per_occupied_tet": npart / occupied}
    # arithmetic roofline of the particle kernel: its FP64 thread instructions
    # (DFMA + DMUL + DADD, counted by ncu on this workload) per launch over the
    # kernel's live duration, against the FP64 FMA rate measured on this GPU
    from paper_2111_12411_gb300.native import measure_alu
    alu = {k: measure_alu(k, local_rank) for k in ("fp64_fma", "fp32_fma", "fp64_div")}
    alu_roof = None
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            ops_pp = tj.get("k_particle_fp64_ops_per_particle_step", {}).get(args.precision)
            pipe_pp = tj.get("k_particle_fp64_pipe_thread_inst_per_particle_step", {}).get(args.precision)
        except (OSError, ValueError, AttributeError):
            ops_pp = pipe_pp = None
        if ops_pp and info.order == 2 and npart == 1_000_000 and args.push == "boris":
            ach = ops_pp * npart / (push_ms * 1e-3)
            alu_roof = {"bound": "alu", "achieved": ach / 1e12, "peak": alu["fp64_fma"] / 1e12,
                        "unit": "T FP64 thread ops/s", "frac": ach / alu["fp64_fma"],
                        "ops_per_particle_step": ops_pp,
                        "fp64_pipe_frac": (pipe_pp * npart / (push_ms * 1e-3) / alu["fp64_fma"]
                                           if pipe_pp else None),
                        "peak_source": "femPIC_measure_alu fp64_fma on this GPU (one DFMA = one op)",
                        "counts": "ncu instruction counts of this kernel on this workload (profiles/traffic.json)"}
    roof_part["alu"] = alu_roof

    # ---- end to end through the C ABI with host buffers ---------------------------------
    e2e = None
    if not args.no_e2e:
        xh = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True).numpy()
        vh = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True).numpy()
        th = torch.empty(npart, dtype=torch.int32, pin_memory=True).numpy()
        eh = torch.empty(info.n1, dtype=torch.float64, pin_memory=True).numpy()
        xh[:] = sim.get("X")
        vh[:] = sim.get("V")
        th[:] = sim.get("TET")
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            sim.set("X", xh)
            sim.set("V", vh)
            sim.set("TET", th)
            sim.step(dt)
            sim.get("X", out=xh)
            sim.get("V", out=vh)
            sim.get("TET", out=th)
            sim.get("E", out=eh)
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = xh.nbytes + vh.nbytes + th.nbytes
        d2h = h2d + eh.nbytes
        e2e = {"value": world * npart * K / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "note": "per step: particle state host->device, one full step, particle state "
                       "and E DOFs device->host, through femPIC_set/step/get straight to and from "
                       "pinned host buffers"}

    result = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            n_s = min(args.cpu_sample, npart)
            ts, cores = oracle_particle_parallel(args.walls, n_s, 1)
            t1 = oracle_particle_sample(cfg, args.cpu_sample_1core, steps=1)
            cpu = {"value": n_s / ts[0], "unit": UNIT, "cores": cores, "kind": "oracle",
                   "cpu": host_cpu(),
                   "sample": f"one particle-loop step (gather, push, walk, deposit, charge) of the "
                             f"first {n_s} of the {npart} particles on the same mesh and seed, split by "
                             f"particles over {cores} host processes, currents summed; the oracle's direct "
                             "field solve is not timed at this size",
                   "single_core": {"value": args.cpu_sample_1core / t1[0], "cores": 1,
                                   "sample": f"the first {args.cpu_sample_1core} particles, one step"}}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision != "mixed" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": workload_name(info.order, npart, args.walls), "precision": args.precision,
                       "push": args.push,
                       "l2": "flushed between steps "
                       "(256 MiB write)", "parallelism": "replicas" if world > 1 else "single GPU",
                       "n_particles": npart, "n_tets": info.n_tets, "n1": info.n1, "n2": info.n2,
                       "device_bytes": int(info.device_bytes),
                       "cg_rtol": args.cg_rtol,
                       "cg_direction_products": "fp32, residual recomputed in fp64 every "
                                                f"{info.cg_replace_period} iterations"
                       if info.cg_fp32_products else "fp64",
                       "cg_preconditioner": (f"Chebyshev smoother of degree {info.cg_smooth_degree} on B^-1 A"
                                             if info.cg_smooth_degree > 1 else "block Jacobi")
                       + f" + auxiliary spaces, {info.aux_cheb_degree} Chebyshev steps"},
            "roofline": roof_pcg if dominant_is_pcg else roof_part,
            "roofline_particle_kernel": roof_part,
            "roofline_cg_kernel": roof_pcg,
            "particle_loop": {"value": world * npart * K / ((acc["particle_ms"]) * 1e-3), "unit": UNIT,
                              "ms_per_step": acc["particle_ms"] / K,
                              "note": "sort + gather/push/walk/deposit/charge only"},
            "field_update": {"ms_per_step": acc["field_ms"] / K, "cg_iterations_per_step": iters,
                             "rhs_ms": acc["rhs_ms"] / K, "pcg_ms": pcg_ms,
                             "bupdate_ms": acc["bupdate_ms"] / K},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(acc["launches"]),
            "alu_peaks_ops_per_s": alu,
            "clocks": clocks,
        }
    sim.close()
    if result is not None and world == 1 and not args.no_extras:
        # the other single-GPU workloads, each a compact sub-record of the same line
        extras_t0 = time.perf_counter()
        result["c3_precision"] = precision_record(args, local_rank, workloads.make_config(2), args.c3_steps, 3,
                                                  args.c3_steps)
        result["batched"] = batched_record(local_rank, args.batched_instances, args.batched_steps, 3)
        result["batched"]["config"]["reduction"] = (
            f"{args.batched_instances} instances x {args.batched_steps} steps of the 64 x 200 batched workload")
        result["serving"] = serving_record(local_rank, args.serving_requests, args.serving_rate, 50, 16, 200.0)
        result["serving"]["config"]["reduction"] = (
            f"{args.serving_requests} of the 512 Poisson requests of the serving workload")
        result["extras_wall_s"] = time.perf_counter() - extras_t0
    if result is not None:
        print(json.dumps(result), flush=True)
    return result


def batched_record(local_rank, n_instances, K, W):
    """Batched workload: uneven box instances advanced together (mixed
    precision, one launch per kernel for all, autotuned launch shapes,
    replayed as one CUDA graph per step) against the plain per-instance FP64
    path (each instance stepped alone, one after the other)."""
    import torch
    import workloads
    from paper_2111_12411_gb300 import Batch, Simulation

    cfgs = workloads.make_batch(n_instances=n_instances, steps=K)
    total_np = sum(len(c["x"]) for c in cfgs)
    out = {"metric": "aggregate particle-steps/s, batched mixed precision vs per-instance FP64",
           "unit": UNIT, "steps": K, "warmup": W, "data": "synthetic",
           "config": {"workload": f"{len(cfgs)} Kuhn-box instances, tets log-uniform 2e3-5e4, p in {{1,2}}, "
                                  "particles log-uniform 1e4-1e6, B0 uniform 0-1 T",
                      "instances": len(cfgs), "particles": total_np,
                      "tets": sum(len(c["tets"]) for c in cfgs),
                      "orders": [c["order"] for c in cfgs]}}
    sims = [Simulation.from_config(c, precision="fp64", device=local_rank) for c in cfgs]
    for _ in range(W):
        for sm, c in zip(sims, cfgs):
            sm.step(c["dt"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = 0
    for _ in range(K):
        for sm, c in zip(sims, cfgs):
            sm.step(c["dt"])
            iters += sm.last_timing()["cg_iterations"]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    for sm in sims:
        sm.close()
    out["per_instance_fp64"] = {"value": total_np * K / t_plain, "ms_per_step": 1e3 * t_plain / K,
                                "cg_iterations_per_instance_step": iters / (K * len(cfgs))}
    sims = [Simulation.from_config(c, precision="mixed", device=local_rank) for c in cfgs]
    batch = Batch(sims)
    dts = np.array([c["dt"] for c in cfgs])
    tune = batch.autotune(dts, steps_per_candidate=1)  # real steps, before the timed region
    batch.step(dts, W)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(dts, K)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    tm = batch.timing()
    out["value"] = total_np * K / t_batch
    out["ms_per_step"] = 1e3 * t_batch / K
    out["batched_mixed"] = {"value": total_np * K / t_batch, "ms_per_step": 1e3 * t_batch / K,
                            "device_ms_per_step": tm["ms"] / K, "cuda_graph": bool(tm["graph"]),
                            "launches_per_step": tm["launches_per_step"], "cg_ctas": tm["cg_ctas"],
                            "autotune": tune}
    out["speedup_batched_vs_per_instance"] = out["value"] / out["per_instance_fp64"]["value"]
    batch.close()
    for sm in sims:
        sm.close()
    return out


def run_batched(args, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    print(json.dumps(batched_record(local_rank, args.instances, args.steps, args.warmup)), flush=True)


def serving_record(local_rank, n_requests, rate, chunk_steps, max_slots, hbm_budget_gb):
    """Serving workload: a Poisson stream of box simulations admitted by HBM
    budget and advanced in chunks with continuous batching."""
    import workloads
    from paper_2111_12411_gb300.serve import Request, Server

    reqs = workloads.make_requests(n_requests=n_requests, rate_hz=rate, chunk_steps=chunk_steps, chunks=(1, 2))
    server = Server(hbm_budget_gb * (1 << 30), max_slots=max_slots, device=local_rank,
                    precision="mixed", result_keys=("E",))
    t_build = time.perf_counter()
    for r in reqs:
        cfg = workloads.build_request(r)
        server.submit(Request(r["id"], cfg, r["arrival"], r["n_chunks"], r["chunk_steps"]))
    t_build = time.perf_counter() - t_build
    server.run()
    rep = server.report()
    return {"metric": "serving: p50/p99 chunk latency and aggregate particle-steps/s", "unit": UNIT,
            "value": rep["particle_steps_per_s_busy"], "data": "synthetic",
            "config": {"workload": f"{len(reqs)} Poisson requests at {rate} Hz, Kuhn boxes 2e3-5e4 "
                                   "tets, p in {1,2}, particles 1e4-4e6, mixed precision",
                       "chunk_steps": chunk_steps, "hbm_budget_gb": hbm_budget_gb,
                       "max_slots": max_slots, "host_input_generation_s": t_build},
            "serving": rep}


def run_serving(args, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    print(json.dumps(serving_record(local_rank, args.requests, args.rate, args.chunk_steps, args.instances,
                                    args.hbm_budget_gb)), flush=True)


def _rooflines(info, acc, crossings, npart, occupied, K, peak, peak_src):
    """HBM rooflines of the CG solve and the particle kernel from K steps of
    library timings (acc: summed last_timing fields) and crossings."""
    iters = acc["cg_iterations"] / K
    pcg_bytes = pcg_bytes_per_iteration(info) * (iters + 1.0)
    pcg_ms = acc["pcg_ms"] / K
    pcg_gbs = pcg_bytes / (pcg_ms * 1e-3) / 1e9
    cross_pp = crossings / (K * max(1, npart))
    pbytes = particle_bytes_per_step(info.order, npart, occupied, cross_pp) * npart
    push_ms = acc["push_ms"] / K
    push_gbs = pbytes / (push_ms * 1e-3) / 1e9
    src = peak_src + " of measured" if "measured" in peak_src else peak_src
    cg = {"kernel": "k_pcg (device PCG, one cooperative launch per step)", "bound": "hbm",
          "achieved": pcg_gbs, "peak": peak, "unit": "GB/s", "frac": pcg_gbs / peak, "traffic": None,
          "peak_source": src, "bytes_per_launch": pcg_bytes, "cg_iterations_per_launch": iters,
          "ms_per_launch": pcg_ms}
    part = {"kernel": "k_particle (gather, push, walk, deposit, charge)", "bound": "hbm",
            "achieved": push_gbs, "peak": peak, "unit": "GB/s", "frac": push_gbs / peak, "traffic": None,
            "peak_source": src, "bytes_per_launch": pbytes, "ms_per_launch": push_ms,
            "crossings_per_particle": cross_pp, "particles_per_occupied_tet": npart / max(1, occupied)}
    return cg, part


def precision_record(args, local_rank, cfg, K, W, err_steps):
    """Mixed precision against FP64 on the same GPU, both forms stepped from the
    same state: each form's throughput (whole step and particle loop, with
    both rooflines), then the relative errors of E, B, x and v of the mixed
    form against the FP64 form after each of err_steps steps, and both forms'
    Gauss and continuity residuals."""
    import torch
    from paper_2111_12411_gb300 import Simulation

    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    npart = len(cfg["x"])
    occupied = len(np.unique(cfg["tet"]))
    peak, peak_src = measured_peaks()

    def rel(a, b):
        nb = float(np.linalg.norm(b))
        return float(np.linalg.norm(a - b)) / nb if nb > 0 else float(np.linalg.norm(a))

    sims = {p: Simulation.from_config(cfg, precision=p, device=local_rank, stream=stream.cuda_stream,
                                      cg_rtol=args.cg_rtol, diagnostics=True) for p in ("fp64", "mixed")}
    info = sims["fp64"].info
    state0 = {k: sims["fp64"].get(k) for k in ("X", "V", "TET", "E", "E_PREV", "B", "DG", "DG_PREV", "RHO")}
    out_forms = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for p, sm in sims.items():
        sm.step(cfg["dt"], W)
        torch.cuda.synchronize(dev)
        t_ms = []
        acc = {k: 0.0 for k in ("particle_ms", "field_ms", "push_ms", "pcg_ms", "cg_iterations", "launches")}
        cross = 0.0
        for _ in range(K):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sm.step(cfg["dt"])
            b.record(stream)
            b.synchronize()
            t_ms.append(a.elapsed_time(b))
            t = sm.last_timing()
            for k in acc:
                acc[k] += t[k]
            cross += sm.diag()["crossings"]
        d = sm.diag()
        from paper_2111_12411_gb300.native import femPIC_get_info
        roof_cg, roof_part = _rooflines(femPIC_get_info(sm.h), acc, cross, npart, occupied, K, peak, peak_src)
        out_forms[p] = {"value": npart * K / (1e-3 * sum(t_ms)), "ms_per_step": sum(t_ms) / K,
                        "particle_loop": {"value": npart * K / (1e-3 * acc["particle_ms"]),
                                          "ms_per_step": acc["particle_ms"] / K,
                                          "note": "sort + gather/push/walk/deposit/charge"},
                        "field_update": {"ms_per_step": acc["field_ms"] / K, "pcg_ms": acc["pcg_ms"] / K,
                                         "cg_iterations_per_step": acc["cg_iterations"] / K},
                        "roofline_particle_kernel": roof_part, "roofline_cg_kernel": roof_cg,
                        "gpu_launches": int(acc["launches"]),
                        "cg_iterations_last_step": d["cg_iterations"]}
        for k, v in state0.items():
            sm.set(k, v)
    errs = []
    for step in range(1, err_steps + 1):
        for sm in sims.values():
            sm.step(cfg["dt"])
        f, m = sims["fp64"], sims["mixed"]
        df, dm = f.diag(), m.diag()
        row = {"step": step}
        for k in ("E", "B", "X", "V"):
            row[k] = rel(m.get(k), f.get(k))
        row["tet_mismatch"] = float(np.mean(m.get("TET") != f.get("TET")))
        for tag, d in (("fp64", df), ("mixed", dm)):
            row[f"gauss_{tag}"] = d["gauss_abs"] / d["gauss_ref"] if d["gauss_ref"] > 0 else d["gauss_abs"]
            row[f"continuity_{tag}"] = (d["continuity_abs"] / d["continuity_ref"]
                                        if d["continuity_ref"] > 0 else d["continuity_abs"])
        errs.append(row)
    out = {"metric": "mixed precision vs FP64 on one GPU: particle-steps/s and per-field relative error",
           "unit": UNIT, "value": out_forms["mixed"]["value"], "steps": K, "warmup": W, "data": "synthetic",
           "config": {"workload": "jittered Kuhn box 37^3 (303918 tets), p=2, "
                                  f"{npart:.0e} electrons in two counter-streaming beams +-2e7 m/s, "
                                  "v_th=1e6 m/s, B0=0".replace("e+0", "e"),
                      "n_particles": npart, "n_tets": info.n_tets, "n1": info.n1, "n2": info.n2,
                      "cg_rtol": args.cg_rtol, "dt": cfg["dt"],
                      "l2": "flushed between timed steps (256 MiB write); particle state alone 0.56 GB"},
           "fp64": out_forms["fp64"], "mixed": out_forms["mixed"],
           "speedup_mixed_vs_fp64": out_forms["mixed"]["value"] / out_forms["fp64"]["value"],
           "errors_mixed_vs_fp64": errs,
           "note": "errors are relative 2-norms of the mixed form against the FP64 form from the same "
                   "initial state; the FP64 form itself matches the oracle to 1e-12 (parity tests)"}
    for sm in sims.values():
        sm.close()
    return out


def run_precision(args, local_rank):
    """Mixed precision against FP64 on the jittered 37^3 Kuhn box (303,918
    tets, p = 2, 10^7 electrons in two counter-streaming beams +-2e7 m/s
    along z, v_th = 1e6 m/s); see precision_record."""
    import torch
    import workloads
    torch.cuda.set_device(local_rank)
    cfg = workloads.make_config(2, n_particles=args.particles)
    print(json.dumps(precision_record(args, local_rank, cfg, args.steps, args.warmup, args.steps)), flush=True)


def run_push(args, local_rank):
    """The paper's Adams-Bashforth push on the quartic path against the Boris
    push on the straight chord, on the drift-tube mesh and beam with the axial
    field lowered to 0.05 T (omega_c dt = 0.29: Adams-Bashforth 4 is stable for
    |omega dt| below about 0.43 on oscillatory motion, the 1 T of the drift-tube
    workload gives 5.9).  Particle loop and whole step, device-timed; charge
    conservation from the library's diagnostics."""
    import torch
    import workloads
    from paper_2111_12411_gb300 import Simulation

    torch.cuda.set_device(local_rank)
    cfg = workloads.make_config(1, n_particles=args.particles)
    cfg["B0"] = (0.0, 0.0, 0.05)
    K, W = args.steps, args.warmup
    npart = len(cfg["x"])
    out = {"metric": "particle-steps/s of the particle loop and the whole step, Adams-Bashforth 4 vs Boris",
           "unit": UNIT, "steps": K, "warmup": W, "data": "synthetic",
           "config": {"workload": "drift tube R=1cm L=10cm, polar Kuhn mesh 24x12x80 (132480 tets), p=2, "
                                  f"{npart} electrons, v_z=3e7 m/s, B0=0.05 T, dt=33.3 ps",
                      "n_particles": npart}}
    for name, push, prec in (("boris_fp64", "boris", "fp64"), ("boris_strict", "boris", "fp64_strict"),
                             ("ab4", "ab4", "fp64")):
        sm = Simulation.from_config(cfg, precision=prec, device=local_rank, push=push, diagnostics=True,
                                    cg_rtol=args.cg_rtol)
        sm.step(cfg["dt"], W)
        torch.cuda.synchronize()
        part = field = 0.0
        worst = 0.0
        cross = 0.0
        for _ in range(K):
            sm.step(cfg["dt"])
            t = sm.last_timing()
            part += t["push_ms"]
            field += t["field_ms"]
            d = sm.diag()
            cross += d["crossings"]
            if d["continuity_ref"] > 0:
                worst = max(worst, d["continuity_abs"] / d["continuity_ref"])
        out[name] = {"particle_kernel_ms": part / K, "particle_steps_per_s": npart * K / (part * 1e-3),
                     "whole_step_ms": (part + field) / K, "crossings_per_particle": cross / (K * npart),
                     "continuity_rel_max": worst}
        sm.close()
    out["value"] = out["ab4"]["particle_steps_per_s"]
    out["ab4_cost_vs_boris_strict"] = out["ab4"]["particle_kernel_ms"] / out["boris_strict"]["particle_kernel_ms"]
    print(json.dumps(out), flush=True)


def run_project(args, local_rank):
    """The divergence-free projection of an impressed flux density (Section
    III-C, eq. conB) on the drift-tube mesh: a quadrupole lens field
    B = grad phi, phi = (G / k^2) sin(k x) sinh(k y) (harmonic, so B is
    divergence- and curl-free; G x y near the axis), G = 1 T/m,
    k = pi / 2 cm (far from polynomial across the 1 cm radius), projected with
    and without Gauss's magnetic law.  Per call: host time of the W3
    operators, device time of the load and the nested CG solve, and the inner
    CG iteration's algorithmic bytes against its device-timed duration (HBM
    roofline)."""
    import torch
    import workloads
    from paper_2111_12411_gb300 import Simulation

    torch.cuda.set_device(local_rank)
    cfg = workloads.make_config(1, n_particles=1000)
    cfg["order"] = args.order
    G, k = 1.0, math.pi / 0.02

    def lens(x):
        return np.stack([G / k * np.cos(k * x[:, 0]) * np.sinh(k * x[:, 1]),
                         G / k * np.sin(k * x[:, 0]) * np.cosh(k * x[:, 1]), 0.0 * x[:, 2]], axis=1)

    sim = Simulation.from_config(cfg, device=local_rank, es_init=False, cg_rtol=args.cg_rtol)
    info = sim.info
    pts = sim.impressed_points()
    Bv = lens(pts)
    peak, peak_src = measured_peaks()
    out = {"metric": "impressed-field projection (eq. conB): device ms per call and inner-CG HBM roofline",
           "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
           "data": "synthetic",
           "config": {"workload": "drift tube R=1cm L=10cm, polar Kuhn mesh 24x12x80 (132480 tets), "
                                  f"p={args.order}, quadrupole lens B = grad((G/k^2) sin(kx) sinh(ky)), "
                                  "G = 1 T/m, k = pi/2cm", "n2": info.n2, "n_points": len(pts),
                      "cg_rtol": args.cg_rtol}}
    traffic_it = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if args.order == 2 and os.path.exists(prof):
        try:
            traffic_it = json.load(open(prof)).get("projection_inner_iteration_dram_bytes_p2")
        except (OSError, ValueError):
            traffic_it = None
    for name, con in (("galerkin", False), ("constrained", True)):
        for _ in range(max(1, args.warmup // 3)):
            sim.set_impressed_B(Bv, constrained=con)
        runs = []
        for _ in range(args.steps):
            runs.append(sim.set_impressed_B(Bv, constrained=con))
        inner_it = sum(r["inner_iterations"] for r in runs)
        inner_ms = sum(r["inner_ms"] for r in runs)
        gbs = runs[0]["bytes_per_inner_iteration"] * inner_it / (inner_ms * 1e-3) / 1e9 if inner_ms > 0 else None
        out[name] = {"device_ms": statistics.median(r["device_ms"] for r in runs),
                     "host_ms": statistics.median(r["host_ms"] for r in runs),
                     "outer_iterations": runs[-1]["outer_iterations"],
                     "inner_iterations": runs[-1]["inner_iterations"],
                     "div_residual": runs[-1]["div_residual"],
                     "inner_iteration_us": 1e3 * inner_ms / max(1, inner_it),
                     "roofline_inner_iteration": {
                         "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak if gbs else None, "traffic": traffic_it,
                         "peak_source": peak_src,
                         "bytes_per_iteration": runs[0]["bytes_per_inner_iteration"]}}
    bi = sim.get("B_IMPRESSED")
    out["value"] = out["constrained"]["device_ms"]
    out["b_impressed_norm"] = float(np.linalg.norm(bi))
    print(json.dumps(out), flush=True)
    sim.close()


def _timed_steps(sm, dt, K, W):
    """W untimed then K timed steps; per-step library timings and diagnostics."""
    import torch
    sm.step(dt, W)
    torch.cuda.synchronize()
    acc = {"particle_ms": 0.0, "field_ms": 0.0, "pcg_ms": 0.0, "cg_iterations": 0.0}
    cont = gauss = 0.0
    for _ in range(K):
        sm.step(dt)
        t = sm.last_timing()
        for k in acc:
            acc[k] += t[k]
        d = sm.diag()
        if d["continuity_ref"] > 0:
            cont = max(cont, d["continuity_abs"] / d["continuity_ref"])
        if d["gauss_ref"] > 0:
            gauss = d["gauss_abs"] / d["gauss_ref"]
    out = {k: v / K for k, v in acc.items()}
    out["step_ms"] = out["particle_ms"] + out["field_ms"]
    out["continuity_rel_max"] = cont
    out["gauss_rel_last"] = gauss
    return out


def run_schemes(args, local_rank):
    """The time schemes of Section III-B / IV-D on the drift-tube workload:
    the trapezoidal rule on [b; e] against the second-order e form with the
    backward-difference (gamma 1.5, beta 1) and Galerkin (gamma 1.5, beta 0.8)
    parameters.  Whole step, CG iterations, Gauss residual after the run."""
    import torch
    import workloads
    from paper_2111_12411_gb300 import Simulation

    torch.cuda.set_device(local_rank)
    cfg = workloads.make_config(1, n_particles=args.particles, walls=args.walls)
    K, W = args.steps, args.warmup
    npart = len(cfg["x"])
    out = {"metric": "particle-steps/s of the whole step per time scheme", "unit": UNIT, "steps": K, "warmup": W,
           "data": "synthetic", "config": {"workload": workload_name(2, npart, args.walls), "cg_rtol": args.cg_rtol}}
    for name, scheme, g, b in (("trapezoid", "trapezoid", 0.5, 0.25), ("backward_difference", "wave", 1.5, 1.0),
                               ("galerkin", "wave", 1.5, 0.8)):
        sm = Simulation.from_config(cfg, device=local_rank, scheme=scheme, gamma=g, beta=b, diagnostics=True,
                                    cg_rtol=args.cg_rtol)
        r = _timed_steps(sm, cfg["dt"], K, W)
        r["particle_steps_per_s"] = npart / (r["step_ms"] * 1e-3)
        out[name] = r
        sm.close()
    out["value"] = out["trapezoid"]["particle_steps_per_s"]
    print(json.dumps(out), flush=True)


def run_species(args, local_rank):
    """Impedance (first-order absorbing) walls and two species, the
    ingredients of the paper's plasma-ball example (Section IV), on a 24^3
    Kuhn box of 1 m, p = 2: electrons (v_th 1e6 m/s) and Sr+ ions (v_th
    1e3 m/s), 5e5 of each, every wall impedance, against the same run with
    PEC walls and one species.  Whole step, CG iterations, continuity."""
    import torch
    import workloads
    from paper_2111_12411_gb300 import Simulation

    torch.cuda.set_device(local_rank)
    n = args.particles or 500_000
    xyz, tets = workloads.kuhn_box(24, 24, 24, jitter=0.1, seed=workloads.configs.SEED0 + 7)
    rng = np.random.default_rng(workloads.configs.SEED0 + 7)
    q_e, m_e = workloads.configs.Q_E, workloads.configs.M_E
    m_sr = 87.62 * 1.66053906660e-27
    h = 1.0 / 24
    omega = 1e6 / h
    n_e = omega * omega * workloads.configs.EPS0 * m_e / (q_e * q_e)
    w = n_e / n
    dt = 0.5 / omega
    xe, te = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    xi, ti = workloads.sample_uniform_in_tets(xyz, tets, n, rng)
    sp = [dict(q=-q_e, m=m_e, weight=w, x=xe, v=workloads.maxwellian(n, 1e6, rng), tet=te),
          dict(q=q_e, m=m_sr, weight=w, x=xi, v=workloads.maxwellian(n, 1e3, rng), tet=ti)]
    tag = np.ones((len(tets), 4), dtype=np.int32)
    K, W = args.steps, args.warmup
    out = {"metric": "particle-steps/s of the whole step, impedance walls and two species vs PEC and one",
           "unit": UNIT, "steps": K, "warmup": W, "data": "synthetic",
           "config": {"workload": f"Kuhn box 24^3 (82944 tets), p=2, {n} electrons + {n} Sr+ ions, "
                                  f"dt={dt:.3g} s, impedance on every wall", "cg_rtol": args.cg_rtol}}
    runs = (("impedance_two_species", dict(species=sp, bface_tag=tag), 2 * n),
            ("pec_electrons", dict(), n))
    for name, kw, npart in runs:
        sm = Simulation(xyz, tets, 2, -q_e, m_e, w, xe, sp[0]["v"], te, device=local_rank, diagnostics=True,
                        cg_rtol=args.cg_rtol, **kw)
        r = _timed_steps(sm, dt, K, W)
        r["particle_steps_per_s"] = npart / (r["step_ms"] * 1e-3)
        r["n_particles"] = npart
        out[name] = r
        sm.close()
    out["value"] = out["impedance_two_species"]["particle_steps_per_s"]
    print(json.dumps(out), flush=True)


def run_oracle_baseline(args):
    """The oracle timed on the host cores, for the CPU baseline table: the
    6^3 box (C1: 1296 tets, p = 1, 10^4 electrons) for all its steps with the
    field solve (single core, numpy/scipy as they stand), and the particle
    loops of the drift tube (10^6 electrons, p = 2) and of the 37^3 box (a
    10^6-particle sample of its 10^7, extrapolated per particle) on one core
    and split over every core.  No GPU is used."""
    import workloads
    from oracle import sim as osim
    out = {"metric": "oracle on the host cores (CPU baseline)", "unit": UNIT, "cpu": host_cpu(),
           "cores": os.cpu_count(), "data": "synthetic"}
    cfg = workloads.make_config(0)
    t0 = time.perf_counter()
    s = osim.Sim(cfg["xyz"], cfg["tets"], cfg["order"], cfg["q"], cfg["m"], cfg["weight"], cfg["B0"],
                 cfg["rho_ion"])
    s.set_particles(cfg["x"], cfg["v"], cfg["tet"])
    s.electrostatic_init()
    t_setup = time.perf_counter() - t0
    steps = cfg["steps"] if args.oracle_c1_steps is None else args.oracle_c1_steps
    t_part = t_field = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        w = s.push_walk(cfg["dt"])
        t1 = time.perf_counter()
        from oracle import fields
        A = fields.system_matrix(s.M, s.K, cfg["dt"], s.scheme, s.gamma, s.beta, s.I)
        r = fields.rhs_trapezoid(s.M, s.K, s.CtM2, s.e, s.b, w["dg"], cfg["dt"], s.I)
        e_new = fields.solve(A, r, s.topo.free1)
        s.b = fields.update_b(s.C, s.b, e_new, s.e, cfg["dt"])
        s.e_prev, s.e = s.e, e_new
        s.x, s.v, s.tet = w["x"], w["v"], w["tet"]
        s.rho = s._measure_rho(s.x, s.tet)
        t_field += time.perf_counter() - t1
        t_part += t1 - t0
    n = len(cfg["x"])
    out["c1"] = {"workload": "6^3 Kuhn box, 1296 tets, p=1, 1e4 electrons", "steps": steps, "cores": 1,
                 "setup_s": t_setup, "particle_loop": n * steps / t_part, "field_solve_s_per_step": t_field / steps,
                 "whole_step": n * steps / (t_part + t_field)}
    for name, idx, n_s in (("c2", 1, 1_000_000), ("c3", 2, 1_000_000)):
        c = workloads.make_config(idx, n_particles=n_s) if idx == 2 else workloads.make_config(idx)
        t1 = oracle_particle_sample(c, min(100_000, n_s), steps=1)[0]
        if idx == 1:
            tp, cores = oracle_particle_parallel("beam", n_s, 1)
        else:
            tp, cores = None, os.cpu_count()
        out[name] = {"workload": c["name"], "particle_loop_1core": min(100_000, n_s) / t1,
                     "particle_loop_all_cores": (n_s / tp[0]) if tp else None, "cores": cores,
                     "sample": f"one step of the first {min(100_000, n_s)} particles (1 core)"
                               + (f"; all {n_s} particles over {cores} processes" if tp else "")}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--precision", default="fp64", choices=("fp64", "fp64_strict", "mixed"))
    ap.add_argument("--particles", type=int, default=None)
    ap.add_argument("--push", default="boris", choices=("boris", "ab4"),
                    help="particle push: Boris on the straight chord, or the paper's Adams-Bashforth 4 "
                         "on the quartic path")
    ap.add_argument("--cg-rtol", type=float, default=1e-12)
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--cpu-sample-1core", type=int, default=100_000)
    ap.add_argument("--ref-sample", type=int, default=400_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sub-records of the default run (37^3 box mixed vs FP64, batched, serving)")
    ap.add_argument("--c3-steps", type=int, default=3)
    ap.add_argument("--oracle-c1-steps", type=int, default=None)
    ap.add_argument("--batched-instances", type=int, default=32)
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--serving-requests", type=int, default=128)
    ap.add_argument("--serving-rate", type=float, default=8.0)
    ap.add_argument("--workload", choices=("tube", "batched", "serving", "precision", "push", "project",
                                           "schemes", "species", "oracle"),
                    default="tube")
    ap.add_argument("--order", type=int, default=2, choices=(1, 2, 3),
                    help="basis order p of the tube and project workloads")
    ap.add_argument("--cg-max-it", type=int, default=2000)
    ap.add_argument("--walls", default="beam", choices=("beam", "reflect"),
                    help="drift tube walls: the beam absorbed at z=L and re-injected at z=0, or reflection")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=2.0)
    ap.add_argument("--chunk-steps", type=int, default=50)
    ap.add_argument("--hbm-budget-gb", type=float, default=200.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "oracle":
        run_oracle_baseline(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_2111_12411_gb300 import build

    def node_barrier():
        import torch.distributed as dist
        dist.barrier()
    build_in_rank_order(local_rank, world, build.build, node_barrier)
    if args.workload == "batched":
        run_batched(args, local_rank)
    elif args.workload == "serving":
        run_serving(args, local_rank)
    elif args.workload == "precision":
        run_precision(args, local_rank)
    elif args.workload == "push":
        run_push(args, local_rank)
    elif args.workload == "project":
        run_project(args, local_rank)
    elif args.workload == "schemes":
        run_schemes(args, local_rank)
    elif args.workload == "species":
        run_species(args, local_rank)
    else:
        run_native(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
