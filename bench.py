#!/usr/bin/env python3
"""Throughput of the online stage (Algorithm 1 stage 2) on one GB300.

Workload: the 192^3-cell model in 8x8x8 = 512 subdomains of 24^3 cells,
m = 8 modes per face (b = 48), k = 16 levels, one 20 Hz Ricker shot, 1024
surface receivers, 4000 leapfrog steps (seeded synthetic layered model with a
Gaussian lens; ``sfm_inputs.config2``).  One bench step is one pass of the
whole online stage: ``sfm_run`` over the 4000 time steps.

Metric: equivalent fine-grid cell-steps/s per shot,
N_cells * nsteps * (dt / dt_fine) * nshots / seconds, for the fastest
precision whose traces stay within 1e-3 (relative L2) of the FP64 run of the
same ROMs.  dt is 0.9x the ROM leapfrog limit (power iteration on the GPU),
dt_fine 0.9x the fine grid's limit from the Gershgorin bound of its operator.

The offline ROM build (GPU, FP64), the source/receiver projection and the
CFL estimate happen before timing.  ``--impl reference`` times the FP64 CPU
oracle (``oracle/``) instead; ``cpu_baseline`` in the default line is the same
oracle timed on a bounded sample."""
from __future__ import annotations

import argparse
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

import sfm_inputs as inputs  # noqa: E402

METRIC = "equivalent fine-grid cell-steps/s per shot at <=1e-3 trace error vs FP64"
UNIT = "cell-steps/s"
GATE = 1e-3
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sfm", choices=["sfm", "reference"])
    ap.add_argument("--nsteps", type=int, default=None, help="time steps per run (default: 4000)")
    ap.add_argument("--precision", default="auto",
                    choices=["auto", "fp32f", "tf32x3", "tf32", "fp32", "fp32fx2", "fp32x2p", "fp32x2", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched config-3 object of the headline line")
    ap.add_argument("--cpu-sample-steps", type=int, default=600)
    ap.add_argument("--workload", default="cfg2", choices=["cfg2", "cfg3", "paper", "paper10", "surrogate"],
                    help="cfg2: 192^3 cells, 512 subdomains, 1 shot (the headline); "
                         "cfg3: 256x256x128 cells, uneven subdomains, 64 shots; "
                         "paper: the 7x7x3 unit-cube layout of the paper's experiment at "
                         "its own m = 25 (b = 150), k = 3, t in [0, 12.5]; paper10: the same "
                         "layout at m = 10, k = 4; surrogate: the learned surrogate "
                         "trained and judged on 24^3 blocks (m = 8, k = 16)")
    ap.add_argument("--sur-train", type=int, default=2000, help="surrogate workload: training blocks")
    ap.add_argument("--sur-test", type=int, default=200, help="surrogate workload: held-out blocks")
    ap.add_argument("--sur-epochs", type=int, default=30)
    ap.add_argument("--shape", default=None,
                    help="fixed stepping block shape 'warps,stages' instead of the autotuner's")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# metric helpers (no method arithmetic)

def fine_dt(p, safety=0.9):
    """0.9 x 2/sqrt(lambda) with lambda the Gershgorin bound of the fine
    operator M^{-1} K (vertex-centred cells: conductance h/4 per edge per
    cell, lumped mass h^3/(8c^2) per corner): every node's row sum times two
    over its mass."""
    h = p.h
    inv = h ** 3 / (8.0 * p.c ** 2)
    m = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1))
    g = np.zeros_like(m)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                m[dz:dz + p.nz, dy:dy + p.ny, dx:dx + p.nx] += inv
                g[dz:dz + p.nz, dy:dy + p.ny, dx:dx + p.nx] += 3 * h / 4.0   # 3 edges per corner
    lam = float(np.max(2.0 * g / m))
    return safety * 2.0 / np.sqrt(lam)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.f.flush()

    def summary(self):
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nme, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM}, "fallback"


def max_over_ranks(x, dist, device):
    """Largest value of x over the ranks of the process group (x itself
    without one): the job's time is its slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms, world):
    """Units all ranks processed per second when each of ``world`` replicas
    processes ``units_per_rank`` in ``ms`` milliseconds (the slowest)."""
    return units_per_rank * world / (ms * 1e-3)


def face_modes(p):
    """Modes per (subdomain, face) of a problem: a shared face carries the
    smaller of its two subdomains' m, an outer face its own (the layout rule
    of the face basis); faces ordered -x, +x, -y, +y, -z, +z."""
    ncx, ncy, ncz = len(p.xcuts) - 1, len(p.ycuts) - 1, len(p.zcuts) - 1
    m = np.asarray(p.m_sub).reshape(ncz, ncy, ncx)
    out = np.zeros((p.nsub, 6), dtype=int)
    for iz in range(ncz):
        for iy in range(ncy):
            for ix in range(ncx):
                s = ix + ncx * (iy + ncy * iz)
                for f, (dx, dy, dz) in enumerate(((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                                                  (0, 0, -1), (0, 0, 1))):
                    jx, jy, jz = ix + dx, iy + dy, iz + dz
                    inside = 0 <= jx < ncx and 0 <= jy < ncy and 0 <= jz < ncz
                    out[s, f] = min(m[iz, iy, ix], m[jz, jy, jx]) if inside else m[iz, iy, ix]
    return out


def algorithmic_bytes_per_step(p, nshots, receiver_numbers, word):
    """Bytes one time step must move (the roofline's per-step figure): once
    per step the coefficient blocks (Gamma_1..k and Gammahat_2..k, each
    b(b+1)/2 numbers, packed symmetric or triangular factor), the face blocks
    H_f and the receiver rows (``receiver_numbers`` in all); per shot U and
    delta read and written and the face data written and read back.
    ``word`` = (bytes per block number, bytes per other number)."""
    wk, ws = word
    mf = face_modes(p)
    b = mf.sum(axis=1)
    k = np.asarray(p.k_sub)
    blocks = int(((2 * k - 1) * b * (b + 1) // 2).sum())
    other = int((mf * (mf + 1) // 2).sum() + receiver_numbers)
    per_shot = int((4 * k * b + 2 * b).sum())
    return blocks * wk + (other + nshots * per_shot) * ws


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline and --impl reference)

def oracle_sample(nsteps_sample):
    """The config-2 stepping workload (same geometry, b, k, receivers) with
    ROM coefficients the oracle builds for a uniform 3000 m/s medium on the
    same grid (one distinct subdomain build): the cost of the stepping does
    not depend on the coefficients' values."""
    from oracle import pipeline
    p = inputs.config2()
    p.c = np.full_like(p.c, 3000.0)
    rs = pipeline.build(p)
    dt = pipeline.rom_dt(rs)
    return p, rs, dt, fine_dt(p)


def time_oracle(p, rs, dt, dtf, nsteps_sample):
    from oracle import coupled
    w = inputs.wavelet_samples(p, dt, nsteps_sample)
    t0, c0 = time.perf_counter(), time.process_time()
    coupled.step_structured(rs, dt, nsteps_sample, w)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    ncell = p.nx * p.ny * p.nz
    value = ncell * nsteps_sample * (dt / dtf) * rs.nshots / wall
    return value, wall, max(1, round(cpu / wall))


def reference_arm(args, rank, world):
    if rank != 0:
        return
    if args.workload != "cfg2":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm is sized for the "
                          "config-2 workload; the other workloads are timed on the GPU only"}))
        return
    p, rs, dt, dtf = oracle_sample(args.cpu_sample_steps)
    ns = args.cpu_sample_steps
    for _ in range(args.warmup):
        time_oracle(p, rs, dt, dtf, ns)
    vals, walls, cores = [], [], 1
    for _ in range(args.steps):
        v, wall, cores = time_oracle(p, rs, dt, dtf, ns)
        vals.append(v)
        walls.append(wall)
    value = statistics.mean(vals)
    sample = (f"config-2 stepping (512 subdomains, b=48, k=16, 1024 receivers, 1 shot), "
              f"{ns} of its time steps per bench step, oracle-built ROMs of a uniform "
              f"3000 m/s medium on the same grid")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": p.name, "sample_time_steps": ns},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------

MODES = ("fp32f", "tf32x3", "tf32", "fp32", "fp32fx2", "fp32x2p", "fp32x2")
DTYPE = {"fp32f": "f32", "tf32x3": "tf32x3", "tf32": "tf32", "fp32": "f32", "fp32fx2": "f32x2",
         "fp32x2p": "f32x2", "fp32x2": "f32x2", "fp64": "f64"}
# bytes per number: (S-fraction blocks or their factors, everything else)
WORD = {"fp32f": (4, 4), "tf32x3": (4, 4), "tf32": (4, 4), "fp32": (4, 4), "fp32fx2": (4, 8),
        "fp32x2p": (8, 8), "fp32x2": (8, 8), "fp64": (8, 8)}
KERNEL = {"tf32x3": "panel_kernel", "tf32": "panel_kernel", "fp32x2p": "panel2_kernel"}
# FP32 operations of one compensated two-float term g x in the two-float
# panel products (two-product 2, two-sum 6, error sums 2, cross terms 2)
X2_TERM_OPS = 12


def build_workload(sfm, h, p, workload):
    """Offline stage on the GPU (not timed by the metric): ROMs, projections,
    depth cut (config 3), CFL step.  Returns (dt, nsteps, dt_fine, report,
    depth_cut, build seconds)."""
    t0 = time.perf_counter()
    sfm.sfm_set_model(h, p.c, p.h, p.xcuts, p.ycuts, p.zcuts)
    rep = sfm.sfm_build_roms(h, p.m_sub, p.k_sub, p.sigma)
    sfm.sfm_project_sources(h, p.src_xyz, p.src_width)
    sfm.sfm_project_receivers(h, p.rec_xyz)
    depth_cut = None
    if workload == "cfg3":
        # the deepest fractions of this workload run past FP64's range: keep
        # each subdomain's usable depth (the rest of the run uses it)
        depth, ncut = sfm.sfm_cut_depth(h, p.nsub, 1e-13)
        depth_cut = {"tau": 1e-13, "levels_cut": int(ncut),
                     "subdomains_cut": int((depth < p.k_sub).sum())}
        p.k_sub = depth.astype(p.k_sub.dtype)
    lam, dtc = sfm.sfm_cfl_dt(h, 1000)
    sfm.sfm_free_build(h)              # the Krylov bases are not needed any more
    build_s = time.perf_counter() - t0
    dt = p.dt_safety * dtc
    nsteps = p.nsteps if p.nsteps else int(np.ceil(p.meta["t_end"] / dt))
    return dt, nsteps, fine_dt(p), rep, depth_cut, build_s


def measure_workload(sfm, torch, h, p, args, dt, nsteps, stream, local, dist, world, warmup, steps,
                     e2e_runs, force=None, also=()):
    """Precision gate, block shape, timed runs (device events, L2 flushed
    between runs, clocks sampled) and the end-to-end rate of one workload.
    ``also``: further modes timed beside the chosen one (reported, not
    chosen)."""
    nshots, nrec = p.nshots, p.nrec
    wav = torch.tensor(inputs.wavelet_samples(p, dt, nsteps), dtype=torch.float64, device="cuda")
    tr = torch.empty((nshots, nrec, nsteps + 1), dtype=torch.float64, device="cuda")
    modes = {"fp32f": sfm.SFM_FP32F, "tf32x3": sfm.SFM_TF32X3, "tf32": sfm.SFM_TF32,
             "fp32": sfm.SFM_FP32, "fp32fx2": sfm.SFM_FP32FX2, "fp32x2p": sfm.SFM_FP32X2P,
             "fp32x2": sfm.SFM_FP32X2,
             "fp64": sfm.SFM_FP64}

    def run(prec):
        _, ms = sfm.sfm_run(h, prec, dt, nsteps, None, nshots, nrec,
                            device_ptrs=(wav.data_ptr(), tr.data_ptr()))
        return ms

    # FP64 reference of the same ROMs, then the precision gate
    run(sfm.SFM_FP64)
    torch.cuda.synchronize()
    ref = tr.cpu().numpy()
    errors = {"fp64": 0.0}
    for name in MODES:
        if name in KERNEL and nshots < 16 and name != force:
            # the panel modes step 16 shots at a time: with fewer shots they
            # do the full panel's work for a fraction of it (not a candidate)
            errors[name] = None
            continue
        try:
            run(modes[name])
            torch.cuda.synchronize()
            errors[name] = rel_l2(tr.cpu().numpy(), ref)
        except sfm.SfmError as e:
            errors[name] = float("inf") if e.code == sfm.SFM_ERR_UNSTABLE else None
    if force:
        chosen = force
    else:
        chosen = next(n for n in ("fp32f", "tf32x3", "fp32", "fp32fx2", "fp32x2p", "fp32x2", "fp64")
                      if errors.get(n) is not None and errors[n] <= GATE)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    timed = {}
    for name in [chosen] + [a for a in also if a != chosen]:
        prec = modes[name]
        if args.shape:
            fixed = [int(v) for v in args.shape.split(",")]
            tune = (fixed[0], fixed[1], None)
            sfm.sfm_debug_set(h, 3, fixed[0])
            sfm.sfm_debug_set(h, 4, fixed[1])
        else:
            tune = sfm.sfm_autotune(h, prec, 200 if nsteps >= 200 else nsteps)
        for _ in range(warmup):
            run(prec)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        kern_ms = []
        with Clocks(local) as clk:
            torch.cuda.synchronize()
            wall0 = time.perf_counter()
            for i in range(steps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                kern_ms.append(run(prec))
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            wall = time.perf_counter() - wall0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        timed[name] = {"ms": max_over_ranks(statistics.mean(step_ms), dist, "cuda"),
                       "kernel_ms": statistics.mean(kern_ms), "launches": sfm.sfm_last_launches(h) * steps,
                       "clocks": clk.summary(), "wall": wall,
                       "block_shape": {"consumer_warps": tune[0], "ring_stages": tune[1],
                                       "probe_us_per_time_step": tune[2]}}
    # end to end through the public API with host buffers (H2D of the
    # wavelet and D2H of the traces inside the timed region)
    host_w = inputs.wavelet_samples(p, dt, nsteps)
    host_tr = np.empty((nshots, nrec, nsteps + 1))
    e2e_t = []
    for _ in range(max(1, e2e_runs)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sfm.sfm_run(h, modes[chosen], dt, nsteps, host_w, nshots, nrec, traces=host_tr)
        e2e_t.append(time.perf_counter() - t1)
    return chosen, errors, timed, statistics.mean(e2e_t), host_w.nbytes, host_tr.nbytes


def alu_peak(clock_mhz):
    """FP32 operations per second of the whole GPU: 152 SMs x 128 FP32 lanes
    x the SM clock (an FMA counts as one operation)."""
    return 152 * 128 * clock_mhz * 1e6


def roofline_of(p, name, t, nsteps, pk, pk_kind, traffic):
    word = WORD[name]
    bytes_step = algorithmic_bytes_per_step(p, p.nshots, receiver_row_numbers(p), word)
    achieved = bytes_step * nsteps / (t["kernel_ms"] * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
           "peak_source": f"{pk_kind} HBM copy",
           "kernel": KERNEL.get(name, "step_kernel"),
           "kernel_ms": t["kernel_ms"], "bytes_per_time_step": bytes_step}
    if name == "fp32x2p":
        # compensated CUDA-core products: bound by FP32 issue, not by bytes
        b = face_modes(p).sum(axis=1)
        k = np.asarray(p.k_sub)
        terms = float(((2 * k - 1) * b * b).sum()) * p.nshots
        ops = terms * X2_TERM_OPS * nsteps
        clk = (t.get("clocks") or {}).get("sm_mhz") or 2070.0
        peak = alu_peak(clk) / 1e12
        ach = ops / (t["kernel_ms"] * 1e-3) / 1e12
        out = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
               "frac": ach / peak, "traffic": traffic,
               "peak_source": f"152 SMs x 128 FP32 lanes x {clk:.0f} MHz (FP32 operations, FMA = 1)",
               "kernel": "panel2_kernel", "kernel_ms": t["kernel_ms"],
               "two_float_terms_per_time_step": terms, "fp32_ops_per_term": X2_TERM_OPS,
               "hbm": {"achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                       "frac": achieved / pk["hbm_gbs"], "bytes_per_time_step": bytes_step}}
    return out


def cpu_baseline_run(threads, sample_steps):
    """The oracle's stepping on a bounded sample, in a child process whose
    BLAS/OpenMP pools are set to ``threads`` before NumPy loads (the child
    never touches the GPU).  Returns (value, wall seconds, cores used)."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[var] = str(threads)
    code = ("import json, bench; p, rs, dt, dtf = bench.oracle_sample({n}); "
            "v, w, c = bench.time_oracle(p, rs, dt, dtf, {n}); print(json.dumps([v, w, c]))").format(n=sample_steps)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"oracle baseline failed: {r.stderr[-500:]}")
    v, w, c = json.loads(r.stdout.strip().splitlines()[-1])
    return v, w, c


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1406_6923_gb300 import sfm

    if args.workload == "surrogate":
        surrogate_experiment(sfm, torch, args)
        return
    makers = {"cfg2": inputs.config2, "cfg3": inputs.config3,
              "paper": lambda: inputs.paper_layout(m=25, k=3),       # the paper's m and n, b = 150
              "paper10": lambda: inputs.paper_layout(m=10, k=4)}
    p = makers[args.workload]()
    stream = torch.cuda.current_stream()
    h = sfm.sfm_create(local)
    sfm.sfm_set_stream(h, stream.cuda_stream)
    dt, nsteps, dtf, rep, depth_cut, build_s = build_workload(sfm, h, p, args.workload)
    if args.nsteps:
        nsteps = args.nsteps
    chosen, errors, timed, e2e_s, h2d, d2h = measure_workload(
        sfm, torch, h, p, args, dt, nsteps, stream, local, dist, world, args.warmup, args.steps, args.steps,
        force=None if args.precision == "auto" else args.precision,
        also=("fp32fx2",) if (args.workload == "cfg2" and not args.no_extra) else ())
    sfm.sfm_destroy(h)
    t = timed[chosen]
    ms = t["ms"]
    nshots = p.nshots
    ncell = p.nx * p.ny * p.nz
    bw = face_modes(p).sum(axis=1)
    widths = int(bw[0]) if bw.min() == bw.max() else [int(bw.min()), int(bw.max())]
    kk = np.asarray(p.k_sub)
    levels = int(kk[0]) if kk.min() == kk.max() else [int(kk.min()), int(kk.max())]
    value = whole_job_rate(ncell * nsteps * (dt / dtf) * nshots, ms, world)
    e2e_val = ncell * nsteps * (dt / dtf) * nshots / e2e_s * world
    pk, pk_kind = peaks()
    traffic = read_traffic() if (args.workload == "cfg2" and chosen == "fp32f") else None
    roof = roofline_of(p, chosen, t, nsteps, pk, pk_kind, traffic)
    if roof["bound"] == "hbm":
        # the factored FP32 coefficient set of config 2 stays in L2 after the
        # first time step: its own roof, measured here
        l2 = sfm.sfm_probe_read_gbs(local, 32 << 20, 64)
        roof["l2"] = {"achieved": roof["achieved"], "peak": l2, "unit": "GB/s",
                      "frac": roof["achieved"] / l2,
                      "peak_source": "measured here (sfm_probe_read_gbs): one launch reading a 32 MB "
                                     "buffer held in L2 64 times, 16-byte L2-cached loads, CUDA events"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "cfg2":
        ncores = os.cpu_count() or 1
        v_all, w_all, c_all = cpu_baseline_run(ncores, args.cpu_sample_steps)
        v_one, w_one, c_one = cpu_baseline_run(1, args.cpu_sample_steps)
        cpu = {"value": v_all, "unit": UNIT, "cores": c_all, "kind": "oracle",
               "sample": (f"config-2 stepping, {args.cpu_sample_steps} of its time steps, "
                          f"oracle-built ROMs of a uniform 3000 m/s medium on the same grid "
                          f"(identical stepping cost), BLAS/OpenMP pools of {ncores} threads "
                          f"on a host of {ncores} cores, {w_all:.1f} s"),
               "nproc": ncores, "one_core": {"value": v_one, "cores": c_one, "seconds": w_one}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE[chosen], "data": "synthetic",
           "config": {"workload": p.name, "cells": ncell, "subdomains": p.nsub,
                      "b": widths, "k": levels,
                      "shots": nshots, "receivers": p.nrec, "time_steps": nsteps,
                      "precision": chosen, "trace_err_vs_fp64": errors,
                      "dt": dt, "dt_fine": dtf, "dt_ratio": dt / dtf,
                      "conservative_value": ncell * nsteps * nshots / (ms * 1e-3) * world,
                      "l2": "256 MB buffer written between timed iterations",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "offline_build_s": build_s, "build": rep, "depth_cut": depth_cut,
                      "block_shape": t["block_shape"]},
           "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
           "gpu_launches": t["launches"], "clocks": t["clocks"], "wall_s_timed": t["wall"]}

    if "fp32fx2" in timed and chosen != "fp32fx2":
        # the FP32-target mode (FP32 factor bytes, two-float state) on the
        # same workload
        tx = timed["fp32fx2"]
        err = errors.get("fp32fx2")
        out.setdefault("extra", {})["fp32fx2"] = {
            "value": whole_job_rate(ncell * nsteps * (dt / dtf) * nshots, tx["ms"], world),
            "ms_per_step": tx["ms"], "trace_err_vs_fp64": err,
            "within_1e-5": err is not None and err <= 1e-5,
            "roofline": roofline_of(p, "fp32fx2", tx, nsteps, pk, pk_kind, None),
            "block_shape": tx["block_shape"], "clocks": tx["clocks"],
            "gpu_launches": tx["launches"]}
    if args.workload == "cfg2" and world == 1 and not args.no_extra:
        out.setdefault("extra", {})["cfg3"] = batched_extra(sfm, torch, args, local, pk, pk_kind)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_extra(sfm, torch, args, local, pk, pk_kind):
    """The batched workload (256 x 256 x 128 cells, 495 uneven subdomains,
    64 shots, 3000 steps) measured beside the headline: its gated precision
    and the multi-shot tensor-core panel mode (SFM_TF32X3), each with 3
    warm-up and 2 timed runs, L2 flushed between runs."""
    p = inputs.config3()
    stream = torch.cuda.current_stream()
    h = sfm.sfm_create(local)
    sfm.sfm_set_stream(h, stream.cuda_stream)
    dt, nsteps, dtf, rep, depth_cut, build_s = build_workload(sfm, h, p, "cfg3")
    chosen, errors, timed, e2e_s, h2d, d2h = measure_workload(
        sfm, torch, h, p, args, dt, nsteps, stream, local, None, 1, 3, 2, 1, also=("tf32x3", "fp32x2"))
    sfm.sfm_destroy(h)
    ncell = p.nx * p.ny * p.nz
    rate = lambda ms: ncell * nsteps * (dt / dtf) * p.nshots / (ms * 1e-3)
    t = timed[chosen]
    res = {"workload": p.name, "cells": ncell, "subdomains": p.nsub, "shots": p.nshots,
           "receivers": p.nrec, "time_steps": nsteps, "depth_cut": depth_cut, "offline_build_s": build_s,
           "precision": chosen, "value": rate(t["ms"]), "unit": UNIT, "ms_per_step": t["ms"],
           "trace_err_vs_fp64": errors, "roofline": roofline_of(p, chosen, t, nsteps, pk, pk_kind, None),
           "block_shape": t["block_shape"], "clocks": t["clocks"],
           "e2e": {"value": ncell * nsteps * (dt / dtf) * p.nshots / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}}
    if "fp32x2" in timed and chosen != "fp32x2":
        # the single-shot two-float kernel on the same workload (every shot
        # its own unit, every block read once per shot)
        tq = timed["fp32x2"]
        res["fp32x2_single_shot_kernel"] = {
            "value": rate(tq["ms"]), "ms_per_step": tq["ms"], "trace_err_vs_fp64": errors.get("fp32x2"),
            "roofline": roofline_of(p, "fp32x2", tq, nsteps, pk, pk_kind, None),
            "block_shape": tq["block_shape"], "clocks": tq["clocks"]}
    if "tf32x3" in timed and chosen != "tf32x3":
        tp = timed["tf32x3"]
        err = errors.get("tf32x3")
        res["tf32x3_panel"] = {"value": rate(tp["ms"]), "ms_per_step": tp["ms"], "trace_err_vs_fp64": err,
                               "passes_gate": err is not None and err <= GATE,
                               "roofline": roofline_of(p, "tf32x3", tp, nsteps, pk, pk_kind, None),
                               "block_shape": tp["block_shape"], "clocks": tp["clocks"]}
    return res


def ntd_frequencies(f_peak, count=16, eta_hz=4.0, band=2.5):
    """lambda_i = (eta + i w_i)^2, w_i = 2 pi f_i, f_i evenly spaced in
    (0, band * f_peak], eta = 2 pi eta_hz: the frequencies the surrogate's
    NtD maps are judged at."""
    f = band * f_peak * np.arange(1, count + 1) / count
    return (2 * np.pi * eta_hz + 2j * np.pi * f) ** 2


def surrogate_experiment(sfm, torch, args):
    """The learned surrogate at the size of the surrogate workload (24^3-cell
    blocks, m = 8, k = 16): exact ROMs of the training and test blocks from
    the GPU builder, the decoder fit, FP32 training on the GPU, the NtD-map
    error at 16 frequencies of the BF16 network on the held-out blocks (and
    of the decoder's mean ROM, the baseline), then the offline stage of a
    model tiled by held-out blocks with the surrogate and exact fallback at
    several tolerances against the plain build: time per block and trace
    error of the FP64 stepping.  Prints one JSON line."""
    from paper_1406_6923_gb300 import surrogate as sur
    n, m, k, f_peak = 24, 8, 16, 20.0
    b, code = 6 * m, 64
    sigma = inputs.default_sigma(f_peak, 8.0)
    ntr, nte = args.sur_train, args.sur_test
    blocks = inputs.surrogate_blocks(ntr + nte, n=n)
    h = sfm.sfm_create(0)
    t0 = time.perf_counter()
    sets, per_block = sur.build_sets(h, blocks, 10.0, m, k, sigma)
    sfm.sfm_destroy(h)
    build_wall = time.perf_counter() - t0
    dev = "cuda"
    nb = len(blocks)
    sets_d = torch.tensor(sets.reshape(nb, -1), device=dev)
    raw = torch.empty((nb, sfm.raw_size(b, k)), dtype=torch.float64, device=dev)
    sfm.sfm_raw_encode(0, nb, b, k, sets_d.data_ptr(), raw.data_ptr())
    net = sfm.sfm_net_create(0, n, 16, 32, 64, 1024, code, 1)
    nparams = sfm.sfm_net_params(net).size
    codes = torch.empty((ntr, code), dtype=torch.float32, device=dev)
    t1 = time.perf_counter()
    sfm.sfm_net_fit_decoder(net, b, k, raw.data_ptr(), ntr, iters=4, seed=7, codes_ptr=codes.data_ptr())
    fit_s = time.perf_counter() - t1
    c = torch.tensor(np.asarray(blocks, np.float32), device=dev)
    t1 = time.perf_counter()
    losses = sur.train(torch, net, c[:ntr].contiguous(), codes, epochs=args.sur_epochs, batch=32, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    lams = ntd_frequencies(f_peak)
    exact = sets_d[ntr:].contiguous()
    pred = sur.predict_sets(torch, net, code, c[ntr:].contiguous(), exact, bf16=True)
    e_net = sfm.sfm_ntd_error(0, nte, b, k, pred.data_ptr(), exact.data_ptr(), lams).max(axis=1)
    zero = torch.zeros((nte, code), dtype=torch.float32, device=dev)
    mean = exact.clone()
    sfm.sfm_net_decode(net, zero.data_ptr(), nte, mean.data_ptr())
    e_mean = sfm.sfm_ntd_error(0, nte, b, k, mean.data_ptr(), exact.data_ptr(), lams).max(axis=1)
    # the offline stage of a model of held-out blocks: plain vs surrogate
    side = 4
    idx = np.arange(ntr, ntr + side ** 3) % nb
    cm, xc, yc, zc, order = sur.tile_blocks(blocks[idx])
    nsub = len(order)
    msub, ksub = np.full(nsub, m), np.full(nsub, k)
    centre = lambda i, j, l: [(i + 0.5) * n * 10.0, (j + 0.5) * n * 10.0, (l + 0.5) * n * 10.0]
    src = np.array([centre(1, 1, 1)])
    rec = np.array([centre(i, 2, 2) for i in range(side)])
    exact_mask = np.zeros(nsub, dtype=np.int32)
    for x in np.concatenate([src, rec]):
        i, j, l = (int(v // (n * 10.0)) for v in x)
        exact_mask[i + side * (j + side * l)] = 1
    hp = sfm.sfm_create(0)                  # the plain ROM set
    sfm.sfm_set_model(hp, cm, 10.0, xc, yc, zc)
    tp = time.perf_counter()
    sfm.sfm_build_roms(hp, msub, ksub, sigma)
    plain_s = time.perf_counter() - tp
    sfm.sfm_project_sources(hp, src, 10.0)
    sfm.sfm_project_receivers(hp, rec)
    _, dtc_p = sfm.sfm_cfl_dt(hp, 1000)
    hh = sfm.sfm_create(0)                  # the surrogate ROM sets
    sfm.sfm_set_model(hh, cm, 10.0, xc, yc, zc)
    nst = 600
    tolerances = []
    for tol in (1e-3, 1e-2, 1e-1, float("inf")):
        ts = time.perf_counter()
        srep, _ = sfm.sfm_build_roms_surrogate(hh, net, msub, ksub, sigma, tol, exact=exact_mask)
        wall = time.perf_counter() - ts
        sfm.sfm_project_sources(hh, src, 10.0)
        sfm.sfm_project_receivers(hh, rec)
        _, dtc_s = sfm.sfm_cfl_dt(hh, 1000)
        # both sets stepped at 0.9 of the smaller of their two CFL limits
        dt = 0.9 * min(dtc_p, dtc_s)
        w = inputs.ricker(np.arange(nst) * dt, f_peak)[None]
        row = {"nt_tol": tol, "accepted": srep["accepted"], "fallback": srep["fallback"],
               "served": srep["eligible"], "gate_err_median": srep["sigma_err_median"],
               "build_s": wall, "build_s_per_block": wall / nsub,
               "surrogate_pass_s": srep["seconds_surrogate"], "exact_pass_s": srep["seconds_exact"],
               "cfl_ratio_to_plain": dtc_s / dtc_p}
        try:
            ref, _ = sfm.sfm_run(hp, sfm.SFM_FP64, dt, nst, w, 1, len(rec))
            got, _ = sfm.sfm_run(hh, sfm.SFM_FP64, dt, nst, w, 1, len(rec))
            row["trace_err_vs_plain"] = rel_l2(got, ref)
        except sfm.SfmError as e:
            row["trace_err_vs_plain"] = None
            row["run_error"] = str(e)
        tolerances.append(row)
    sfm.sfm_destroy(hh)
    sfm.sfm_destroy(hp)
    sfm.sfm_net_destroy(net)
    out = {"workload": "surrogate_24c_m8_k16", "train_blocks": ntr, "test_blocks": nte,
           "network": {"params": int(nparams), "channels": [16, 32, 64], "hidden": 1024, "code": code,
                       "train": "FP32, Adam 1e-3, batch 32", "epochs": args.sur_epochs,
                       "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
                       "train_s": train_s, "inference": "BF16 weights and activations, FP32 accumulation"},
           "builder": {"blocks": nb, "wall_s": build_wall, "blocks_per_s": nb / build_wall,
                       "s_per_block_in_build": per_block},
           "decoder_fit_s": fit_s,
           "ntd_error_16_freqs": {"network_median": float(np.median(e_net)),
                                  "network_p90": float(np.percentile(e_net, 90)),
                                  "network_max": float(e_net.max()),
                                  "mean_rom_median": float(np.median(e_mean))},
           "offline_stage_4x4x4": {"plain_build_s": plain_s, "plain_s_per_block": plain_s / nsub,
                                   "exact_marked": int(exact_mask.sum()), "time_steps": nst,
                                   "by_tolerance": tolerances}}
    print(json.dumps(out), flush=True)


def receiver_row_numbers(p):
    """Numbers in all receiver rows: one row of k*b per (receiver, subdomain)
    pair, a receiver on a node shared by several subdomains having one pair
    per subdomain."""
    xs = [np.asarray(p.xcuts), np.asarray(p.ycuts), np.asarray(p.zcuts)]
    ncx, ncy = len(p.xcuts) - 1, len(p.ycuts) - 1
    kb = face_modes(p).sum(axis=1) * np.asarray(p.k_sub)
    n = 0
    for x in p.rec_xyz:
        nodes, w = inputs.trilinear_node_weights(x, p.h, p.nx, p.ny, p.nz)
        subs = set()
        for nd in nodes:
            cand = [np.nonzero((c[:-1] <= nd[a]) & (nd[a] <= c[1:]))[0] for a, c in enumerate(xs)]
            for i in cand[0]:
                for j in cand[1]:
                    for k in cand[2]:
                        subs.add(int(i + ncx * (j + ncy * k)))
        n += int(sum(kb[s] for s in subs))
    return n


def read_traffic():
    """DRAM bytes per launch of the stepping kernel from the committed ncu
    summary, when it was taken on the current kernel source (the kernel's
    own file and the number policies; else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_kernel_config2.md")
    src = b""
    for f in ("step_kernel.cuh", "numeric.cuh"):
        with open(os.path.join(ROOT, "paper_1406_6923_gb300", "csrc", f), "rb") as fh:
            src += fh.read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- traffic"):
            k, v = line.split(":", 1)
            vals[k.strip("- ").strip()] = v.strip()
    if vals.get("traffic_source_hash") != digest:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


if __name__ == "__main__":
    main()
