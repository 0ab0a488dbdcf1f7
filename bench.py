"""Benchmark: BSSN RK4 grid-point updates per second on one GB300.

Workload (default): Brill-Lindquist two-puncture data (bare masses 0.5 at
x = +-1.5) on a 128^3 grid over [-8, 8]^3, 8th-order finite differences,
5 ghost zones with a static outer boundary, 1+log slicing, Gamma-driver shift
(eta = 2), Kreiss-Oliger eps = 0.1, dt = 0.25 h, double precision. One step
is one full RK4 step (4 x ghost fill + difference tables + fused
right-hand-side/dissipation/stage kernel) over every interior point; the
metric counts interior points advanced per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one independent replica per GPU (the method's
single-GPU path does not exchange data; weak scaling). --impl reference
times the CPU oracle (test infrastructure) on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BSSN RK4 grid-point updates/sec at 1 GB300, FP64 vs FP32/learned, at stated error"
UNIT = "grid-point updates/s"
N, G, ORDER, LO, HI = 128, 5, 8, -8.0, 8.0
WORKLOAD = ("Brill-Lindquist two punctures (m=0.5 at x=+-1.5), 128^3 on [-8,8]^3, 8th-order FD, 5 ghosts, static "
            "boundary, 1+log + Gamma-driver (eta=2), KO eps=0.1, dt=0.25h, FP64, RK4")

# Measured copy bandwidth and dense BF16 GEMM rate of this GPU type
# (absent on machines where they were not measured).
try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        MEASURED = json.load(_f)
except (OSError, ValueError):
    MEASURED = {}

# DRAM traffic of the fused stage kernel per launch, from one ncu capture of
# the same source (profiles/k_stage_fp64_bl64.md); ignored when the kernel
# source has changed. Captured at 64^3 (262,144 points: 921.1 MB read + 797.5
# MB written per launch, 6.56 kB per point at 4 blocks/SM, rows traversed in
# bricks) and scaled to 128^3 by the point count, since the traffic is per
# point (state, tables and the per-thread stack).
TRAFFIC = {"src_sha": "64481867ccf4c0a5", "bytes_per_launch_128": (920577024 + 797818880) * 128 ** 3 / 64 ** 3}
# FP64 pipe utilisation of the same launch (sm__pipe_fp64_cycles_active,
# percent of peak over active cycles) and the FP64 instructions it executed
# per interior point (smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul}
# _pred_on.sum / 64^3), for the same source.
FP64_PIPE_BUSY = {"src_sha": "64481867ccf4c0a5", "pct_of_active_cycles": 82.56,
                  "dfma_per_point": 636223488 / 64 ** 3, "dadd_per_point": 409468928 / 64 ** 3,
                  "dmul_per_point": 101187584 / 64 ** 3}
# The same for the tiled FP32-RHS stage kernel k_stage32t<8,0> as the bench
# times it (per-stage calls; the roofline's 864 B per point is the average of
# the four stages): the mean of the four stages' launches at 64^3, 1043.6 MB
# read and written in all, 0.995 kB per point and launch
# (profiles/k_stage32t_fp32_bl64.md), scaled to 128^3 by the point count.
TRAFFIC_F32 = {"src_sha": "c9578cbd115078fd",
               "bytes_per_launch_128": (150967552 + 75629568 + 206530560 + 83616512 + 206648064 + 83771904 +
                                        197803520 + 38672384) / 4 * 128 ** 3 / 64 ** 3}
N_SM = 152
FP64_FMA_PER_CLK_SM = 2


# DRAM traffic of one k_cfd_mass_rb iteration at 256^3 (ncu dram__bytes_read.sum
# + dram__bytes_write.sum), for the source it was taken on.
CFD_TRAFFIC = {"src_sha": "1559830c488ce0a5", "bytes_per_launch": 286361600 + 225778176}

# the sources that make up the fused FP64 stage kernel k_stage<8,0,double>
STAGE_SOURCES = ("bssn_common.cuh", "bssn_point.cuh", "bssn_kernels.cuh", "bssn_order.cu", "bssn_bounds.cuh")
# and the tiled FP32-RHS stage kernel k_stage32t<8,0>
STAGE32_SOURCES = ("bssn_common.cuh", "bssn_point.cuh", "bssn_stage32.cuh", "bssn_stage32_types.h", "bssn_stage32.cu", "bssn_cvt.cuh",
                   "bssn_tc.cuh", "bssn_bounds.cuh")


def src_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1307_6488_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_src_sha():
    return src_sha(STAGE_SOURCES)


def kernel32_src_sha():
    return src_sha(STAGE32_SOURCES)


# Stencil applications per interior point and right-hand side (counts of the
# method, not of any implementation): first derivatives of W, gt_ij (6), K,
# Gt^i (3), alpha, beta^i (3) along 3 axes; diagonal and mixed second
# derivatives of W, gt_ij, alpha, beta^i; upwinded advection of all 24
# variables along 3 axes, summed over the axes (2 adds per variable).
N_FIRST, N_SECOND, N_MIXED, N_ADV, N_ADV_SUM = 45, 33, 33, 72, 48


def stage_bytes(prec, stage, order=8, whole_step=False):
    """Algorithmic DRAM bytes per interior point of one fused RK4 stage
    (0..3): every array the stage must read or write once. Both forms read
    the stage input and y0, read the accumulator from stage 1 on, write it
    up to stage 2 and write the next state; FP64 reads the first-difference
    tables (x and y differences of the 11 variables with mixed derivatives,
    order/2 doubles each), FP32-RHS reads the single-precision input, its
    D_x / D_y tables (22 floats) and W in double precision instead of the
    double-precision input; inside bssn_rk4_step the FP32-RHS stages 0..2
    also write the next stage's single-precision input."""
    nv = 24
    common = nv * 8 * (1 + (stage > 0) + (stage < 3) + 1)  # y0, acc read, acc written, ynext
    if prec == "fp64":
        return nv * 8 + 2 * 11 * (order // 2) * 8 + common
    b = nv * 4 + 22 * 4 + 8 + common
    if whole_step and stage < 3:
        b += nv * 4
    return b


def mean_stage_bytes(prec, order=8):
    return sum(stage_bytes(prec, s, order) for s in range(4)) / 4


def executed_fp64(stage_ms, pts, sm_mhz, per_clk, sha):
    """FP64 instructions the fused stage kernel executes per point (ncu
    counts for this source, else None) and their issue rate per SM clock as a
    fraction of the measured FP64 FMA rate per SM clock."""
    if FP64_PIPE_BUSY["src_sha"] != sha:
        return None
    c = FP64_PIPE_BUSY
    inst = c["dfma_per_point"] + c["dadd_per_point"] + c["dmul_per_point"]
    per_clk_run = inst * pts / (stage_ms * 1e-3) / (N_SM * sm_mhz * 1e6)
    return {"fp64_inst_per_point": inst, "fp64_flop_per_point": 2 * c["dfma_per_point"] + c["dadd_per_point"]
            + c["dmul_per_point"], "inst_per_clk_sm": per_clk_run, "frac_of_measured_issue_rate": per_clk_run / per_clk}


def algorithmic_flops(order=ORDER):
    """Flops per interior point and RK4 stage, from the oracle's per-stencil
    counts (pinned against hand counts in tests/test_flop_counts.py): each
    mixed derivative counted as one first-derivative stencil applied to shared
    first derivatives, the oracle's pointwise algebra, Kreiss-Oliger for the
    24 variables plus one add each to put it into the right-hand side, and
    the stage update (acc += b dt k, ynext = y0 + c dt k: 4 per variable)."""
    import oracle
    c = oracle.flop_counts(order)
    gather = (N_FIRST * c["first"] + N_SECOND * c["second"] + N_MIXED * c["first"] + N_ADV * c["upwind_dir"]
              + N_ADV_SUM)
    per_rhs = gather + c["rhs_algebra"]
    ko = 24 * (c["ko_var"] + 1)
    rk = 24 * 4
    return dict(rhs=per_rhs, ko=ko, rk=rk, total=per_rhs + ko + rk, gather=gather, first=c["first"],
                second=c["second"], adv_dir=c["upwind_dir"], algebra=c["rhs_algebra"],
                mixed_tensor=c["mixed_tensor"], n=(N_FIRST, N_SECOND, N_MIXED, N_ADV))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 4 + i and s[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BSSN_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ reference arm (CPU oracle)
def oracle_block(n=32):
    """The workload's central n^3 block (same spacing, order, gauge and
    dissipation as the 128^3 grid, static boundary from its own t = 0 ghosts)
    for the CPU oracle: (state, h, dt, params)."""
    import oracle
    from paper_1307_6488_gb300 import inputs
    h = (HI - LO) / N
    lo = -n * h / 2
    u, _ = inputs.brill_lindquist(n, G, lo=lo, hi=-lo)
    p = oracle.Params(fd_order=ORDER, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    return u, h, 0.25 * h, p


def cpu_oracle_rate(budget_s=15.0, n=32, max_steps=None):
    """Oracle RK4 steps of the same workload (8th order BL, static boundary)
    on an n^3 block of the [-8,8]^3 domain spacing; returns updates/s,
    steps, seconds, threads."""
    import oracle
    u, h, dt, p = oracle_block(n)
    oracle.rk4_step(u, G, h, dt, p, bc=1, ghost_src=u)  # warm the library
    t0 = time.perf_counter()
    steps = 0
    y = u
    while True:
        y = oracle.rk4_step(y, G, h, dt, p, bc=1, ghost_src=u)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n ** 3 * steps / el, steps, el, threads


def cpu_oracle_rate_single_thread(budget_s=4.0, n=16):
    """The same oracle timing with one OpenMP thread, in a child process (the
    thread count is fixed when the oracle library loads); returns
    (updates/s, steps, seconds) or None if the child fails."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r = bench.cpu_oracle_rate(budget_s=%r, n=%d); print(json.dumps(r[:3]))" % (ROOT, budget_s, n))
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        return tuple(json.loads(out.stdout.strip().splitlines()[-1]))
    except Exception:  # noqa: BLE001 - a baseline that could not be taken is reported as missing
        return None


def cpu_oracle_gauge_wave_24(want_state=True):
    """The 24^3 gauge-wave configuration in full on the oracle: 10 RK4 steps
    (4th order, 3 ghosts, periodic, 1+log + Gamma-driver, KO 0.1, dt = dx/4,
    A = 0.01 plus 1e-10 seeded noise). Returns (final state or None,
    updates/s, seconds, threads)."""
    import oracle
    from paper_1307_6488_gb300 import inputs
    u, h = inputs.gauge_wave(24, 3, amplitude=0.01, noise=1e-10, seed=1307)
    p = oracle.Params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    dt = 0.25 * h
    oracle.rk4_step(u, 3, h, dt, p, bc=0)  # warm the library
    t0 = time.perf_counter()
    y = u
    for _ in range(10):
        y = oracle.rk4_step(y, 3, h, dt, p, bc=0)
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return (y if want_state else None), 10 * 24 ** 3 / el, el, threads


def cpu_oracle_gauge_wave_24_single_thread():
    """The same on one OpenMP thread, in a child process; (updates/s, seconds)
    or None."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r = bench.cpu_oracle_gauge_wave_24(False); print(json.dumps(r[1:3]))" % (ROOT,))
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        return tuple(json.loads(out.stdout.strip().splitlines()[-1]))
    except Exception:  # noqa: BLE001 - a baseline that could not be taken is reported as missing
        return None


def run_reference(args):
    # under torchrun only rank 0 times the oracle; the other ranks leave at
    # once (no process group: nothing is exchanged)
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    n = 32
    # input built and the library loaded before the clock starts; the timed
    # region is exactly K oracle RK4 steps, each on the previous one's result
    u, h, dt, p = oracle_block(n)
    y = u
    for _ in range(args.warmup):
        y = oracle.rk4_step(y, G, h, dt, p, bc=1, ghost_src=u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = oracle.rk4_step(y, G, h, dt, p, bc=1, ghost_src=u)
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = n ** 3 * args.steps / el
    sample = (f"one oracle RK4 step per step on the central {n}^3 block of the 128^3 workload (same spacing, "
              f"order, gauge, KO; static boundary from the block's own t = 0 ghosts); updates/s of that block")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_grid": n,
                       "sampling": f"a {n}^3 block of the 128^3 grid: updates/s is per interior point, so the "
                                   f"rate carries over; the oracle's cost per point does not depend on the grid "
                                   f"size"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
TENSORS = [[0], list(range(1, 7)), [7], list(range(8, 14)), list(range(14, 17)), [17], list(range(18, 21)),
           list(range(21, 24))]


def tensor_rel_err(got, want, g):
    """Max over variables of |got - want| normalised by the largest component
    of the same tensor field (interior points)."""
    gi = got[:, g:-g, g:-g, g:-g].reshape(24, -1)
    wi = want[:, g:-g, g:-g, g:-g].reshape(24, -1)
    mag = np.max(np.abs(wi), axis=1)
    scale = np.zeros_like(mag)
    for grp in TENSORS:
        scale[grp] = np.max(mag[grp])
    return np.max(np.abs(gi - wi), axis=1) / np.maximum(scale, 1e-300)


def run_gpu(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1307_6488_gb300 import binding as B
    from paper_1307_6488_gb300 import inputs

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    flops = algorithmic_flops(ORDER)
    n = args.grid
    u, h = inputs.brill_lindquist(n, G, lo=LO, hi=HI)
    grid = B.make_grid(n, ghost=G, dx=h)
    p = B.make_params(fd_order=ORDER, ko_eps=0.1, lapse=0, shift=0, shift_coeff=0.75, eta=2.0, advect_gauge=1)
    dt = 0.25 * h
    state0 = B.upload(u, grid, device=dev)
    ghost_src = state0.clone()
    ya = B.alloc_state(grid, device=dev)
    yb = B.alloc_state(grid, device=dev)
    acc = B.alloc_state(grid, device=dev)
    work = B.alloc_work(grid, p, device=dev)
    rates = None if (args.profile or args.corrector_only or args.amr_only or args.cfd_only) else B.probe_fp_rates()

    def run_form(prec, sample_clocks, whole_step=False):
        """Warm-up and timed RK4 steps of one form. Default: each stage through
        its own calls (ghost fill, tables, fused stage) with CUDA events around
        every fused-stage launch inside the timed region. whole_step: one
        bssn_rk4_step call per step (the FP32 form then converts the state to
        single precision once per step, each stage leaving the next its
        single-precision input); the fused stage is then timed on two more
        steps made of single calls (without those extra stores)."""
        state = state0.clone()
        launches = [0]
        bufs3 = B.alloc_state(grid, device=dev, n=3) if whole_step else None

        def staged(ev=None, y=None):
            y = state if y is None else y
            ys = y
            outs = [ya, yb, ya, y]
            for s in range(4):
                B.fill_ghosts(grid, 1, ghost_src, ys)
                B.diff_tables(grid, p, prec, ys, work)
                if ev is not None:
                    ev.append(torch.cuda.Event(enable_timing=True))
                    ev[-1].record(stream)
                B.rk4_stage_fused(grid, p, prec, s, dt, y, ys, acc, outs[s], work)
                if ev is not None:
                    ev.append(torch.cuda.Event(enable_timing=True))
                    ev[-1].record(stream)
                ys = outs[s]
            B.fill_ghosts(grid, 1, ghost_src, y)
            launches[0] += 13 if prec == B.FP64 else 17

        def step(ev=None):
            if not whole_step:
                staged(ev)
                return
            B.rk4_step(grid, p, prec, dt, 1, ghost_src, state, bufs3, work)
            # FP32: one conversion, 4 x (ghost fill, tables, fused stage), final ghost fill
            launches[0] += 13 if prec == B.FP64 else 14

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        launches[0] = 0
        ev = []
        barrier(world)
        torch.cuda.synchronize()
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(ev)
        t1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__()
        barrier(world)
        ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
        timed_launches = launches[0]
        if whole_step:
            spare = state.clone()  # the timed state stays at its step count
            for _ in range(2):
                staged(ev, spare)
            torch.cuda.synchronize()
            del spare
        launches[0] = timed_launches
        stage_ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(len(ev) // 2)]
        l2, mx, st = B.constraints(grid, p, state, work)
        alg, _, _ = B.algebraic_constraints(grid, p, state, work)
        return dict(state=state, ms=ms, stage_ms=float(np.mean(stage_ms)), launches=launches[0], l2=l2, alg=alg,
                    clocks=clk.summary() if clk else None)

    def run_batched(prec):
        """192 seeded uneven patches (sides 16..96, 4 ratio-2 levels around the
        punctures, 4 ghosts, tricubic Brill-Lindquist fill), 4th order, one
        graph launch per RK4 step over all patches. The FP32-RHS form runs the
        single grids' TMA-tiled stage kernel over the patches."""
        patches = inputs.patch_tree()
        pb = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
        blocks = []
        for q in patches:
            gq = B.make_grid(*q["n"], ghost=4, dx=q["h"])
            w = torch.from_numpy(inputs.bl_conformal_tricubic(q["n"], 4, q["h"], q["origin"])).to(dev)
            st = B.alloc_state(gq, device=dev)
            v4 = B.view4(st, gq)
            v4[inputs.IDX["W"]] = w
            v4[inputs.IDX["alpha"]] = w
            for i in range(3):
                v4[inputs.IDX["gt11"] + inputs.SYM[i][i]] = 1.0
            blocks.append((gq, st, st.clone()))
        dtb = 0.25 * min(q["h"] for q in patches)
        nlev = len({float(q["h"]) for q in patches})
        t_tune = time.perf_counter()
        plan = B.plan_create(blocks, pb, prec, 1)
        t_tune = time.perf_counter() - t_tune
        try:
            pts, tiles, shapes = B.plan_info(plan, len(blocks))
            for _ in range(args.warmup):
                B.batch_step(plan, dtb)
            torch.cuda.synchronize()
            barrier(world)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                B.batch_step(plan, dtb)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        finally:
            B.plan_destroy(plan)
        del blocks
        torch.cuda.empty_cache()
        return {"value": world * pts * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
                "patches": len(patches), "interior_points": int(pts), "tiles": int(tiles),
                "tile_shapes_chosen": np.bincount(shapes, minlength=7).tolist(), "plan_create_s": t_tune,
                "fd_order": 4, "dt": dtb, "graph_launches_per_step": 1,
                # FP64: per stage ghost fill, tables, stage (persistent kernels over all
                # patches); FP32-RHS: ghost fill, single-precision copy, tables, and one
                # tiled stage launch per spacing; then a final ghost fill
                "kernel_nodes_per_step": 13 if prec == B.FP64 else 4 * (3 + nlev) + 1,
                "stage_kernel": "kb_stage<4,double> (persistent, autotuned tiles)" if prec == B.FP64 else
                                "k_stage32t_batch<4> (TMA-staged 8x4x4 tiles, one launch per spacing)"}

    def run_amr(prec):
        """Berger-Oliger hierarchy around the two punctures: 5 levels, 96^3
        cells per level on levels 0-3 (h = 1 .. 1/8, each the middle half of
        the one above, 8 patches each) and two 48^3 boxes at h = 1/16 around
        the punctures; [-48, 48]^3 with a radiative outer boundary; 8th order,
        5 ghosts, dt0 = h0/4 with every finer level subcycled by 2. One step
        is one coarse step (one graph launch): 16.8 M interior updates."""
        ncells, xlo, h0, geo = inputs.bl_hierarchy()
        pa = B.make_params(fd_order=ORDER, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
        states, grids = [], []
        for (lev, o, nn) in geo:
            gq = B.make_grid(*nn, ghost=G, dx=h0 / 2 ** lev)
            st = B.upload(inputs.brill_lindquist_box(o, nn, G, h0 / 2 ** lev, xlo), gq, device=dev)
            states.append(st)
            grids.append(gq)
        t_c = time.perf_counter()
        h = B.amr_create([(lev, o, nn, gq.var_stride, st, None) for (lev, o, nn), gq, st in zip(geo, grids, states)],
                         ncells, xlo, h0, G, 2, 0.25 * h0, pa, prec)
        t_c = time.perf_counter() - t_c
        try:
            for _ in range(args.warmup):
                B.amr_step(h)
            torch.cuda.synchronize()
            barrier(world)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                B.amr_step(h)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
            info = B.amr_info(h)
        finally:
            B.amr_destroy(h)
        fine = len(geo) - 2  # first box on the finest level
        wk = B.alloc_work(grids[fine], pa, device=dev)
        l2, mx, st = B.constraints(grids[fine], pa, states[fine], wk)
        del states, wk
        torch.cuda.empty_cache()
        return {"value": world * info["updates_per_step"] * args.steps / (ms * 1e-3), "unit": UNIT,
                "ms_per_step": ms / args.steps, "levels": info["levels"], "patches": len(geo),
                "updates_per_coarse_step": info["updates_per_step"], "graph_nodes_per_step": info["graph_nodes"],
                "ghost_entries": info["entries"], "create_s": t_c, "fd_order": ORDER, "boundary": "radiative",
                "ham_l2_finest_after": float(l2[0]), "steps_after": args.warmup + args.steps,
                "workload": "Brill-Lindquist (m=0.5 at x=+-1.5), [-48,48]^3, 5 ratio-2 levels (96^3 cells on "
                            "levels 0-3, 2 x 48^3 at h=1/16), Berger-Oliger subcycling, RK4, 8th order, 5 ghosts"}

    def run_rk3(prec):
        """The paper's own integrator (third-order Runge-Kutta, Shu-Osher
        SSP form) on the same 128^3 workload: three fused stages per step,
        no accumulator. Timed through bssn_rk3_step."""
        st = state0.clone()
        bufs = torch.empty(2 * 24 * grid.var_stride, dtype=torch.float64, device=dev)
        wk = B.alloc_work(grid, p, prec, device=dev)
        for _ in range(args.warmup):
            B.rk3_step(grid, p, prec, dt, 1, ghost_src, st, bufs, wk)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            B.rk3_step(grid, p, prec, dt, 1, ghost_src, st, bufs, wk)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        l2, _, _ = B.constraints(grid, p, st, wk)
        del bufs, wk
        return {"value": world * n ** 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "stages_per_step": 3,
                "ham_l2_after": float(l2[0]), "steps": args.steps + args.warmup}

    def run_gauge_wave_24():
        """The small periodic configuration: 24^3 gauge wave (A = 0.01 along x,
        seeded 1e-10 noise, seed 1307) on [-0.5, 0.5]^3, 4th order, 3 ghosts,
        1+log + Gamma-driver, KO 0.1, dt = dx/4, 10 RK4 steps through
        bssn_rk4_step. 13,824 points: launch-latency bound, so the 10 steps
        (130 launches) are also replayed as one captured CUDA graph."""
        ug, hg = inputs.gauge_wave(24, 3, amplitude=0.01, noise=1e-10, seed=1307)
        gq = B.make_grid(24, ghost=3, dx=hg)
        pg = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
        st = B.upload(ug, gq, device=dev)
        s0 = st.clone()
        bufs = torch.empty(3 * 24 * gq.var_stride, dtype=torch.float64, device=dev)
        wk = B.alloc_work(gq, pg, device=dev)
        dtg = 0.25 * hg

        def ten():
            for _ in range(10):
                B.rk4_step(gq, pg, B.FP64, dtg, 0, None, st, bufs, wk)

        for _ in range(args.warmup):
            ten()
        torch.cuda.synchronize()
        reps = 5
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ten()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_eager = e0.elapsed_time(e1) / reps
        # the same 10 steps captured once and replayed
        cg = torch.cuda.CUDAGraph()
        st.copy_(s0)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            ten()  # warm the side stream before capture
        stream.wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(cg, stream=side):
            ten()
        for _ in range(args.warmup):
            cg.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            cg.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_graph = e0.elapsed_time(e1) / reps
        # the same 10 steps on the oracle (all host cores and one), and the
        # GPU's 10-step state against the oracle's
        st.copy_(s0)
        ten()
        torch.cuda.synchronize()
        got = B.download(st, gq)
        want, cpu_rate, cpu_s, cpu_threads = cpu_oracle_gauge_wave_24()
        one = cpu_oracle_gauge_wave_24_single_thread()
        del bufs, wk
        return {"value": world * 10 * 24 ** 3 / (ms_graph * 1e-3), "unit": UNIT, "ms_per_10_steps_graph": ms_graph,
                "ms_per_10_steps_eager": ms_eager, "launches_per_10_steps": 130,
                "cpu_oracle": {"value": cpu_rate, "unit": UNIT, "seconds": cpu_s, "cores": cpu_threads,
                               "single_thread": None if one is None else {"value": one[0], "seconds": one[1]}},
                "gpu_vs_oracle_after_10_steps_max_rel_per_tensor": float(np.max(tensor_rel_err(got, want, 3))),
                "workload": "24^3 gauge wave + 1e-10 noise, periodic, 4th order, 3 ghosts, 10 RK4 steps"}

    def run_paper_shape(nn, lo, hi, prec, method, steps):
        """A uniform Brill-Lindquist grid in one of the paper's own shapes,
        8th order, 5 ghosts, static boundary, timed through bssn_rk3_step
        (method 3, the paper's integrator) or bssn_rk4_step (method 4)."""
        uu, hh = inputs.brill_lindquist(nn, G, lo=lo, hi=hi)
        gq = B.make_grid(nn, ghost=G, dx=hh)
        st = B.upload(uu, gq, device=dev)
        src = st.clone()
        del uu
        bufs = torch.empty((2 if method == 3 else 3) * 24 * gq.var_stride, dtype=torch.float64, device=dev)
        wk = B.alloc_work(gq, p, prec, device=dev)
        stepf = B.rk3_step if method == 3 else B.rk4_step
        dtq = 0.25 * hh
        for _ in range(args.warmup):
            stepf(gq, p, prec, dtq, 1, src, st, bufs, wk)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            stepf(gq, p, prec, dtq, 1, src, st, bufs, wk)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        del st, src, bufs, wk
        torch.cuda.empty_cache()
        return ms

    def run_paper_shapes():
        """The paper's two GPU configurations with Brill-Lindquist data in
        place of its QC-0 data: its single-GPU benchmark, 100^3 evolved
        points + 5 ghosts at 8th order (Sec. 3.4), and its binary-black-hole
        grid, 270^3 points on [-6.75, 6.75]^3, 8th order, RK3 (Sec. 3.3), which
        the paper spread over 27 GPUs and which fits one GB300."""
        out = {}
        ms = run_paper_shape(100, -8.0, 8.0, B.FP64, 3, args.steps)
        rhs_flops = flops["rhs"]
        out["benchmark_100^3_rk3_fp64"] = {
            "value": world * 100 ** 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "rhs_gflops": world * 3 * rhs_flops * 100 ** 3 / (ms * 1e-3) / 1e9,
            "paper_context": "25 GFlop/s on one NVIDIA M2050 (Fermi), same grid shape, McLachlan's own flop count"}
        for prec, name in ((B.FP64, "fp64"), (B.FP32_RHS, "fp32_rhs")):
            ms = run_paper_shape(270, -6.75, 6.75, prec, 3, max(1, min(args.steps, 3)))
            out[f"bbh_270^3_rk3_{name}"] = {"value": world * 270 ** 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                           "paper_context": "27 NVIDIA M2050 GPUs at 90^3 points each"}
        return out

    def run_cfd():
        """The paper's CFD benchmark shape (Sec. 3.2): incompressible Navier-Stokes
        by SOLA in single precision on 256^3 cells, three kernels (velocity,
        4 red-black mass-conservation iterations, boundary after each). Here a
        lid-driven cavity (no-slip walls, lid speed 1, nu = 1e-3, i.e. Re =
        1000 on the unit box), dt = h/4, omega = 1.7, donor fraction 0.3,
        starting from rest. One step is one bssn_cfd_step call."""
        Nc = 256
        hc = 1.0 / Nc
        d = B.make_cfd((Nc, Nc, Nc), hc, (0, 0, 0), nu=1e-3, dt=0.25 * hc, omega=1.7, alpha=0.3, lid=1.0)
        npts = B.cfd_points(d)
        u_, v_, w_, p_ = (torch.zeros(npts, dtype=torch.float32, device=dev) for _ in range(4))
        scratch = torch.zeros(3 * ((npts + 3) // 4 * 4), dtype=torch.float32, device=dev)
        iters = 4
        for _ in range(args.warmup):
            B.cfd_step(d, iters, u_, v_, w_, p_, scratch)
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            B.cfd_step(d, iters, u_, v_, w_, p_, scratch)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps
        # the dominant kernel alone: one fused mass-conservation iteration
        # (both colours), faces alternating between the two sets of arrays,
        # CUDA events on the launching stream
        src, dst = (u_, v_, w_), tuple(scratch[i * ((npts + 3) // 4 * 4):][:npts] for i in range(3))
        ev = []
        for it in range(args.steps):
            ev.append(torch.cuda.Event(enable_timing=True))
            ev[-1].record(stream)
            B.cfd_mass_iteration(d, *src, *dst, p_)
            ev.append(torch.cuda.Event(enable_timing=True))
            ev[-1].record(stream)
            src, dst = dst, src
        torch.cuda.synchronize()
        mass_ms = float(np.mean([ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(len(ev) // 2)]))
        cells = Nc ** 3
        # algorithmic bytes per cell and iteration: u, v, w read and every face
        # written once (12 + 12), p read and written (4 + 4)
        mass_bytes = 32.0 * cells
        hbm = MEASURED.get("hbm_gbs")
        fin = bool(torch.isfinite(u_).all() and torch.isfinite(p_).all())
        umax = float(u_.view(Nc + 2, Nc + 2, Nc + 2)[1:-1, 1:-1, 1:-1].abs().max())  # interior (the lid ghost is 2U - u)
        del u_, v_, w_, p_, scratch
        torch.cuda.empty_cache()
        return {"value": world * cells / (ms * 1e-3), "unit": "cell updates/s", "ms_per_step": ms,
                "mass_iterations_per_step": iters, "gflops_algorithmic": world * 295 * cells / (ms * 1e-3) / 1e9,
                "flops_per_cell_step": 295, "finite": fin, "max_abs_u_interior": umax,
                "roofline": {"bound": "hbm", "kernel": "k_cfd_mass_rb (one red-black iteration in one pass)",
                             "achieved": mass_bytes / (mass_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": (mass_bytes / (mass_ms * 1e-3) / 1e9 / hbm) if hbm else None,
                             "launch_ms": mass_ms, "bytes_per_cell": 32,
                             "traffic": CFD_TRAFFIC["bytes_per_launch"] if CFD_TRAFFIC["src_sha"] == src_sha(
                                 ("bssn_cfd.cu",)) else None},
                "paper_context": "90.5 GFlop/s (Chemora) and 43 GFlop/s (Physis) on one NVIDIA M2050, 256^3, "
                                 "the paper's own flop count",
                "workload": "lid-driven cavity 256^3, FP32, Re 1000, SOLA, 4 mass iterations per step"}

    def run_fp32_config():
        """FP32-RHS against FP64 as stated for that form: throughput of both at
        256^3 (same Brill-Lindquist data, 8th order, g = 5; state 3.6 GB per
        copy), and the accuracy of FP32 against FP64 after 100 RK4 steps at
        96^3 (per-variable max relative error, per-tensor error and the
        Hamiltonian-constraint L2 of each)."""
        out = {}
        for nn, nsteps in ((256, max(1, min(args.steps, 5))),):
            un, hn = inputs.brill_lindquist(nn, G, lo=LO, hi=HI)
            gn = B.make_grid(nn, ghost=G, dx=hn)
            src = B.upload(un, gn, device=dev)
            del un
            bufs = torch.empty(3 * 24 * gn.var_stride, dtype=torch.float64, device=dev)
            wk = B.alloc_work(gn, p, device=dev)
            for name, prec in (("fp64", B.FP64), ("fp32_rhs", B.FP32_RHS)):
                st = src.clone()
                for _ in range(2):
                    B.rk4_step(gn, p, prec, 0.25 * hn, 1, src, st, bufs, wk)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(nsteps):
                    B.rk4_step(gn, p, prec, 0.25 * hn, 1, src, st, bufs, wk)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / nsteps
                out[f"{name}_{nn}^3"] = {"value": nn ** 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                         "steps": nsteps}
                del st
            del src, bufs, wk
            torch.cuda.empty_cache()
        out["fp32_speedup_256^3"] = out["fp32_rhs_256^3"]["value"] / out["fp64_256^3"]["value"]
        na, nst = 96, 100
        ua, ha = inputs.brill_lindquist(na, G, lo=LO, hi=HI)
        ga = B.make_grid(na, ghost=G, dx=ha)
        src = B.upload(ua, ga, device=dev)
        bufs = torch.empty(3 * 24 * ga.var_stride, dtype=torch.float64, device=dev)
        wk = B.alloc_work(ga, p, device=dev)
        res = {}
        for name, prec in (("fp64", B.FP64), ("fp32_rhs", B.FP32_RHS)):
            st = src.clone()
            for _ in range(nst):
                B.rk4_step(ga, p, prec, 0.25 * ha, 1, src, st, bufs, wk)
            torch.cuda.synchronize()
            l2, mx, _ = B.constraints(ga, p, st, wk)
            res[name] = (B.download(st, ga), float(l2[0]))
        a, b = res["fp32_rhs"][0], res["fp64"][0]
        ai = a[:, G:-G, G:-G, G:-G].reshape(24, -1)
        bi = b[:, G:-G, G:-G, G:-G].reshape(24, -1)
        per_var = np.max(np.abs(ai - bi), axis=1) / np.maximum(np.max(np.abs(bi), axis=1), 1e-300)
        out["accuracy_96^3_100_steps"] = {
            "max_rel_per_variable": {v: float(e) for v, e in zip(inputs.VARS, per_var)},
            "max_rel_per_tensor": float(np.max(tensor_rel_err(a, b, G))),
            "ham_l2_fp64": res["fp64"][1], "ham_l2_fp32_rhs": res["fp32_rhs"][1],
            "reference": "the GPU FP64 path (oracle-matched to 1e-12 per right-hand side)"}
        del src, bufs, wk, res
        torch.cuda.empty_cache()
        return out

    def run_learned():
        """Learned half-resolution evolution: train the corrector on pairs the
        plain method generates (64^3 coarse step vs restricted 128^3 fine
        step; Brill-Lindquist data with masses 0.3-0.7 and separations 2-4,
        every fifth trajectory a gauge wave; 4th order), then time learned
        coarse steps (coarse RK4 + correction + Hamiltonian check, fallback
        to the fine method) against the plain fine method over the same
        physical time, and state the error of each against the restricted
        fine solution."""
        from paper_1307_6488_gb300 import learned as LR
        nc, per_traj = 64, 20
        ntraj = max(1, args.learned_pairs // per_traj)
        # trajectory settings only; each problem's initial data is made when
        # its trajectory runs and freed after
        rng = np.random.default_rng(0)
        specs = []
        for i in range(ntraj):
            if i % 5 == 4:
                specs.append(("gw", dict(amplitude=float(rng.uniform(0.02, 0.1)))))
            else:
                m = rng.uniform(0.3, 0.7, 2)
                specs.append(("bl", dict(masses=tuple(m), separation=float(rng.uniform(2, 4)))))
        corr = B.corrector_create(nc, 4, seed=1)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            data = LR.Dataset(corr, nc)
            # normalisation scales from the first (pilot) trajectories, which
            # include a gauge wave; every pair is packed to BF16 as soon as
            # the scales are known, so only packed pairs stay resident. The
            # fine trajectories run in the FP32-RHS form (FP64 state).
            pilot = min(len(specs), 5)
            pending = []
            for i, (kind, kw) in enumerate(specs):
                pr = LR.Problem(kind, nc, **kw)
                ps = LR.trajectory_pairs(LR.Stepper(pr, fine_prec=B.FP32_RHS), per_traj)
                if i >= pilot:
                    data.add(ps, pr.gc)
                    continue
                pending.append((pr, ps))
                if i == pilot - 1:
                    sample = [pp for _, qs in pending for pp in qs[::3]]
                    B.corrector_set_scales(corr, *LR.default_scales(sample, pr.gc))
                    for q, qs in pending:
                        data.add(qs, q.gc)
                    pending = sample = None
            torch.cuda.synchronize()
            t_gen = time.perf_counter() - t0
            t0 = time.perf_counter()
            losses = LR.train(corr, data, epochs=args.learned_epochs, batch=4, lr=1e-3, lr_final=5e-5)
            torch.cuda.synchronize()
            t_train = time.perf_counter() - t0
            train_steps = len(losses)
            del data
            # held-out problems: accuracy over 8 coarse steps
            held = {"bl_m0.45_0.55_d2.7": ("bl", dict(masses=(0.45, 0.55), separation=2.7)),
                    "bl_m0.35_0.65_d3.5": ("bl", dict(masses=(0.35, 0.65), separation=3.5)),
                    "gauge_wave_a0.07": ("gw", dict(amplitude=0.07))}
            acc = {}
            for name, (kind, kw) in held.items():
                st = LR.Stepper(LR.Problem(kind, nc, **kw))
                acc[name] = LR.evaluate(st, corr, 8)
            # throughput: learned coarse step vs two plain fine steps (same dt_c)
            st = LR.Stepper(LR.Problem("bl", nc, masses=(0.45, 0.55), separation=2.7))
            y = st.src_c.clone()
            scratch = torch.empty_like(y)
            fb = 0
            for _ in range(args.warmup):
                fb += LR.learned_step(st, corr, y, scratch=scratch)[0]
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fb += LR.learned_step(st, corr, y, scratch=scratch)[0]
            e1.record(stream)
            torch.cuda.synchronize()
            ms_learned = e0.elapsed_time(e1) / args.steps
            f = st.src_f.clone()
            for _ in range(args.warmup):
                st.fine_step(f)
            e0.record(stream)
            for _ in range(args.steps):
                st.fine_step(f)
                st.fine_step(f)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_fine2 = e0.elapsed_time(e1) / args.steps
            c = st.src_c.clone()
            e0.record(stream)
            for _ in range(args.steps):
                st.coarse_step(c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_coarse = e0.elapsed_time(e1) / args.steps
            # the network alone: one 64^3 inference pass (input copy, 5
            # tensor-core convolutions), inputs resident, passes queued back
            # to back on the stream (the serving call does not wait)
            xb = torch.empty((nc ** 3, 32), dtype=torch.bfloat16, device=dev)
            tb = torch.empty_like(xb)
            B.corrector_pack(corr, st.p.gc, y, y, xb, tb)
            out = torch.empty((nc ** 3, 32), dtype=torch.float32, device=dev)
            for _ in range(args.warmup):
                B.corrector_infer_async(corr, 1, xb, out)
            B.corrector_sync(corr)
            reps = max(10, args.steps)
            e0.record(stream)
            for _ in range(reps):
                B.corrector_infer_async(corr, 1, xb, out)
            e1.record(stream)
            B.corrector_sync(corr)
            ms_forward = e0.elapsed_time(e1) / reps
            mma96 = B.probe_mma_rate(96)
            # the same network on coarse steps in the FP32-RHS form (FP64
            # state, Hamiltonian check and fallback in FP64; the fine
            # reference and the plain fine timing stay FP64)
            acc32 = {}
            for name in ("bl_m0.45_0.55_d2.7", "bl_m0.35_0.65_d3.5"):
                kind, kw = held[name]
                acc32[name] = LR.evaluate(LR.Stepper(LR.Problem(kind, nc, **kw), prec=B.FP32_RHS,
                                                     fine_prec=B.FP64), corr, 8)
            st32 = LR.Stepper(LR.Problem("bl", nc, masses=(0.45, 0.55), separation=2.7), prec=B.FP32_RHS,
                              fine_prec=B.FP64)
            y32 = st32.src_c.clone()
            fb32 = 0
            for _ in range(args.warmup):
                fb32 += LR.learned_step(st32, corr, y32, scratch=scratch)[0]
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                fb32 += LR.learned_step(st32, corr, y32, scratch=scratch)[0]
            e1.record(stream)
            torch.cuda.synchronize()
            ms_learned32 = e0.elapsed_time(e1) / args.steps
            c32 = st32.src_c.clone()
            e0.record(stream)
            for _ in range(args.steps):
                st32.coarse_step(c32)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_coarse32 = e0.elapsed_time(e1) / args.steps
            del st32, y32, c32
        finally:
            B.corrector_destroy(corr)
        torch.cuda.empty_cache()
        nf3 = (2 * nc) ** 3
        # algorithmic network flops per point: 2 x 27 taps x (24x32 + 3 x 32x32 + 32x24) multiply-adds
        net_flops = 2 * 27 * (24 * 32 + 3 * 32 * 32 + 32 * 24)
        conv_tflops = net_flops * nc ** 3 / (ms_forward * 1e-3) / 1e12
        return {"value": 2 * nf3 / (ms_learned * 1e-3), "unit": "fine-grid-equivalent point updates/s",
                "plain_fine_value": 2 * nf3 / (ms_fine2 * 1e-3),
                "speedup_vs_plain_fine": ms_fine2 / ms_learned,
                "ms_learned_step": ms_learned, "ms_two_fine_steps": ms_fine2, "ms_plain_coarse_step": ms_coarse,
                "fallbacks_in_timed_steps": int(fb),
                "on_fp32_rhs_coarse_steps": {
                    "value": 2 * nf3 / (ms_learned32 * 1e-3), "unit": "fine-grid-equivalent point updates/s",
                    "speedup_vs_plain_fine": ms_fine2 / ms_learned32, "ms_learned_step": ms_learned32,
                    "ms_plain_coarse_step": ms_coarse32, "fallbacks_in_timed_steps": int(fb32),
                    "accuracy_8_coarse_steps": acc32,
                    "note": "the network trained above, applied after coarse RK4 steps in the FP32-RHS form; "
                            "errors against the FP64 fine method"},
                "network_forward_ms_64cubed": ms_forward,
                "network_roofline": {"bound": "tensor", "achieved": conv_tflops,
                                     "peak": MEASURED.get("bf16_tflops", 1922.5), "unit": "TFLOP/s",
                                     "frac": conv_tflops / MEASURED.get("bf16_tflops", 1922.5),
                                     "flops_per_point": net_flops,
                                     "peak_source": "measured dense BF16 (cuBLAS burst)",
                                     "mma_n96_ceiling": mma96,
                                     "frac_of_mma_n96_ceiling": conv_tflops / mma96,
                                     "mma_n96_source": "measured rate of back-to-back M=128 N=96 K=16 BF16 tcgen05 "
                                                       "MMAs issued as the convolutions issue them "
                                                       "(bssn_probe_mma_rate)",
                                     "frac_of_dense_bf16": conv_tflops / MEASURED.get("bf16_tflops", 1922.5)},
                "accuracy_8_coarse_steps": acc,
                "accuracy_note": "err_* = RMS over interior points and variables of (x - restricted fine) / "
                                 "per-variable RMS change of the fine solution over the run; ham_* = Hamiltonian "
                                 "constraint L2 (FP64)",
                "training": {"pairs": ntraj * per_traj, "trajectories": ntraj, "epochs": args.learned_epochs,
                             "batch": 4, "adam_steps": train_steps, "loss_first": losses[0],
                             "loss_last20_mean": float(np.mean(losses[-20:])), "gen_s": t_gen, "train_s": t_train,
                             "ms_per_train_step": 1e3 * t_train / max(1, train_steps)},
                "config": "coarse 64^3 / fine 128^3 on [-8,8]^3 (gauge wave [-0.5,0.5]^3), 4 ghosts, 4th order, "
                          "1+log + Gamma-driver, KO 0.1, dt_c = 0.25 h_c, FP64 evolution (training trajectories: "
                          "fine steps in the FP32-RHS form); corrector 5 x conv3d 3^3, 32 channels, GELU (tanh "
                          "form), BF16 tcgen05 with FP32 accumulation; fallback if H L2 > 2x plain coarse"}

    if args.corrector_only:
        # the network's kernels alone on seeded packed data (64^3, batch 4):
        # Adam training steps and single-sample forward passes; for ncu
        nc, S = 64, 4
        corr = B.corrector_create(nc, S, seed=1)
        try:
            gen = torch.Generator(device=dev).manual_seed(0)
            xs = [torch.randn((nc ** 3, 32), device=dev, generator=gen).to(torch.bfloat16) for _ in range(S)]
            ts = [(0.1 * torch.randn((nc ** 3, 32), device=dev, generator=gen)).to(torch.bfloat16) for _ in range(S)]
            for x, t in zip(xs, ts):
                x[:, 24:] = 0
                t[:, 24:] = 0
            out = torch.empty((nc ** 3, 32), dtype=torch.float32, device=dev)
            for _ in range(args.warmup):
                B.corrector_train_step_raw(corr, xs, ts, 1e-4)
                B.corrector_infer_async(corr, 1, xs[0], out)
            B.corrector_sync(corr)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                B.corrector_train_step_raw(corr, xs, ts, 1e-4)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_train = e0.elapsed_time(e1) / args.steps
            e0.record(stream)
            for _ in range(args.steps):
                B.corrector_infer_async(corr, 1, xs[0], out)
            e1.record(stream)
            B.corrector_sync(corr)
            ms_fwd = e0.elapsed_time(e1) / args.steps
            # the same pass waited for after each call, and the training
            # forward pass (hidden pre-activations stored) waited for likewise
            e0.record(stream)
            for _ in range(args.steps):
                B.corrector_infer_async(corr, 1, xs[0], out)
                B.corrector_sync(corr)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_fwd_wait = e0.elapsed_time(e1) / args.steps
            e0.record(stream)
            for _ in range(args.steps):
                B.corrector_forward_raw(corr, 1, xs[0], out)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_fwd_raw = e0.elapsed_time(e1) / args.steps
        finally:
            B.corrector_destroy(corr)
        if rank == 0:
            print(json.dumps({"corrector_only": f"{nc}^3", "batch": S, "ms_per_train_step": ms_train,
                              "ms_per_forward_1_sample": ms_fwd, "ms_per_forward_waited": ms_fwd_wait,
                              "ms_per_forward_raw_waited": ms_fwd_raw}))
        return

    if args.cfd_only:
        res = run_cfd()
        if rank == 0:
            print(json.dumps({"cfd_only": True, **res}))
        return

    if args.batched_only:
        res = {"batched_fp64": run_batched(B.FP64), "batched_fp32_rhs": run_batched(B.FP32_RHS)}
        if rank == 0:
            print(json.dumps({"batched_only": True, **res}))
        return

    if args.learned_only:
        res = run_learned()
        if rank == 0:
            print(json.dumps({"learned_only": True, **res}))
        return

    if args.amr_only:
        # the refined-hierarchy forms alone (for ncu launch lists)
        res = {"amr_fp64": run_amr(B.FP64), "amr_fp32_rhs": run_amr(B.FP32_RHS)}
        if rank == 0:
            print(json.dumps({"amr_only": True, **res}))
        return

    f64 = run_form(B.FP64, not args.profile)
    f32 = run_form(B.FP32_RHS, False, whole_step=True)
    if args.profile:
        # profiling run (small case under ncu): only the two timed step loops
        if rank == 0:
            print(json.dumps({"profile_grid": n, "fp64_stage_ms": f64["stage_ms"], "fp32_stage_ms": f32["stage_ms"]}))
        return
    err32 = tensor_rel_err(B.download(f32["state"], grid), B.download(f64["state"], grid), G)
    batched = {}
    if not args.no_batched:
        batched["batched_fp64"] = run_batched(B.FP64)
        batched["batched_fp32_rhs"] = run_batched(B.FP32_RHS)
    # gravitational-wave extraction (Weyl scalar Psi_4, E, B, invariant) on the
    # evolved 128^3 state, timed like the stage kernel
    vs = grid.var_stride
    wout = torch.empty(16 * vs, dtype=torch.float64, device=dev)
    st = f64["state"]
    origin = (LO + 0.5 * h,) * 3

    def psi4_once():
        B.psi4(grid, p, st, origin, work, psi_re=wout[0:vs], psi_im=wout[vs:2 * vs], inv_re=wout[2 * vs:3 * vs],
               inv_im=wout[3 * vs:4 * vs], E=wout[4 * vs:10 * vs], B=wout[10 * vs:16 * vs])

    for _ in range(args.warmup):
        psi4_once()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        psi4_once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_psi4 = e0.elapsed_time(e1) / args.steps
    batched["psi4_fp64"] = {"ms_per_evaluation": ms_psi4, "points_per_s": n ** 3 / (ms_psi4 * 1e-3),
                            "share_of_rk4_step_if_every_step": ms_psi4 / (ms_psi4 + f64["ms"] / args.steps),
                            "outputs": "Psi_4 (re, im), invariant I (re, im), E_ij, B_ij at every interior point"}
    del wout
    batched["gauge_wave_24"] = run_gauge_wave_24()
    batched["paper_shapes"] = run_paper_shapes()
    if not args.no_cfd:
        batched["cfd_sola_256"] = run_cfd()
    if not args.no_amr:
        batched["amr_fp64"] = run_amr(B.FP64)
        batched["amr_fp32_rhs"] = run_amr(B.FP32_RHS)
    batched["rk3_fp64"] = run_rk3(B.FP64)
    batched["rk3_fp32_rhs"] = run_rk3(B.FP32_RHS)
    if not args.no_fp32_config:
        batched["fp32_rhs_vs_fp64"] = run_fp32_config()
    if not args.no_learned:
        batched["learned_64_from_128"] = run_learned()

    # end to end through the public API with host buffers (pinned): every step
    # uploads its input state, runs one RK4 step (bssn_rk4_step) and reads the
    # result back. The steps are independent problems, so the copies of one
    # step overlap the compute of its neighbours: two device states, uploads
    # and downloads on a copy stream, the step on the compute stream; the
    # timed region spans the first upload to the last download.
    flat_bytes = 24 * grid.var_stride * 8
    h_in = torch.empty(24 * grid.var_stride, dtype=torch.float64, pin_memory=True)
    h_in.copy_(state0.cpu())
    h_out = [torch.empty_like(h_in, pin_memory=True) for _ in range(2)]
    bufs = torch.empty(3 * 24 * grid.var_stride, dtype=torch.float64, device=dev)
    dst = [torch.empty_like(state0) for _ in range(2)]
    cs = torch.cuda.Stream(device=dev)
    e2e_steps = max(2, min(args.steps, 10))

    def e2e_run(nsteps):
        up = [torch.cuda.Event() for _ in range(nsteps)]
        done = [torch.cuda.Event() for _ in range(nsteps)]
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            dst[0].copy_(h_in, non_blocking=True)
            up[0].record(cs)
        for st in range(nsteps):
            if st + 1 < nsteps:
                # the other state was last read by the download of step st - 1,
                # already queued on the copy stream
                with torch.cuda.stream(cs):
                    dst[(st + 1) % 2].copy_(h_in, non_blocking=True)
                    up[st + 1].record(cs)
            stream.wait_event(up[st])
            B.rk4_step(grid, p, B.FP64, dt, 1, ghost_src, dst[st % 2], bufs, work)
            done[st].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(done[st])
                h_out[st % 2].copy_(dst[st % 2], non_blocking=True)
        stream.wait_stream(cs)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    # the downloaded result is the device result
    assert torch.equal(h_out[(e2e_steps - 1) % 2], dst[(e2e_steps - 1) % 2].cpu())

    if rank != 0:
        return
    pts = n ** 3
    value = world * pts * args.steps / (f64["ms"] * 1e-3)
    e2e_value = world * pts * e2e_steps / (e2e_ms * 1e-3)
    achieved = flops["total"] * pts / (f64["stage_ms"] * 1e-3)  # FLOP/s of the fused stage kernel
    # FP64 peak: the FP64 FMA rate per SM clock measured by the probe (SM
    # cycle counter; the unit count gives 2), times the SMs, 2 flop and the
    # median SM clock sampled during the timed region. The probe's own rate
    # per second, at whatever clock it ran, is reported beside it.
    sm_mhz = (f64["clocks"] or {}).get("sm_mhz") or MEASURED.get("sm_max_mhz") or 2070.0
    per_clk = rates["fp64_fma_per_clk_sm"]
    peak = N_SM * per_clk * 2.0 * sm_mhz * 1e6
    peak_nominal = N_SM * FP64_FMA_PER_CLK_SM * 2.0 * sm_mhz * 1e6
    peak_probe = 2.0 * rates["fp64_fma_per_s"]
    sha = kernel_src_sha()
    traffic = TRAFFIC["bytes_per_launch_128"] if TRAFFIC["src_sha"] == sha and n == N else None
    cpu_rate, cpu_steps, cpu_s, cpu_threads = cpu_oracle_rate(budget_s=args.cpu_budget, n=32)
    cpu_one = cpu_oracle_rate_single_thread()
    achieved32 = flops["total"] * pts / (f32["stage_ms"] * 1e-3)
    peak32 = 2.0 * rates["fp32_fma_per_s"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": f64["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N else WORKLOAD.replace("128^3", f"{n}^3"), "grid": n, "fd_order": ORDER, "ghost": G, "precision": "fp64",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (each state copy %.0f MB > 129 MB)" % (flat_bytes / 1e6)},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_stage<8,0,double> (fused RHS+KO+RK stage)",
                     "flops_per_point": flops["total"], "stage_ms": f64["stage_ms"],
                     "peak_source": f"measured {per_clk:.3f} FP64 FMA/clock/SM (probe, SM cycle counter) x "
                                    f"{N_SM} SMs x 2 flop at the sampled median SM clock {sm_mhz:.0f} MHz",
                     "peak_nominal": peak_nominal / 1e12,
                     "peak_probe": peak_probe / 1e12,
                     "peak_probe_sm_mhz": rates["sm_mhz_fp64_fma"],
                     "frac_of_probe": achieved / peak_probe,
                     # the HBM side of the same kernel: algorithmic bytes per point and stage,
                     # averaged over the four stages (stage_bytes): ys 192, difference tables
                     # 704, y0 192, acc read 144 and written 144, ynext 192
                     "hbm": {"bytes_per_point_stage": mean_stage_bytes("fp64"),
                             "achieved_gbs": mean_stage_bytes("fp64") * pts / (f64["stage_ms"] * 1e-3) / 1e9,
                             "frac": (mean_stage_bytes("fp64") * pts / (f64["stage_ms"] * 1e-3) / 1e9 /
                                      MEASURED["hbm_gbs"])
                             if MEASURED.get("hbm_gbs") else None},
                     "fp64_pipe_busy_ncu": FP64_PIPE_BUSY if FP64_PIPE_BUSY["src_sha"] == sha else None,
                     # what the kernel executes (ncu instruction counts of the same source): FP64
                     # instructions per point and stage, and their rate per SM clock against the
                     # probe's measured FMA rate per SM clock (the FP64 pipe's issue ceiling)
                     "executed": executed_fp64(f64["stage_ms"], pts, sm_mhz, per_clk, sha)},
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                         "sample": f"{cpu_steps} oracle RK4 step(s) of the same workload on a 32^3 block "
                                   f"({cpu_s:.1f} s)",
                         "single_thread": None if cpu_one is None else {
                             "value": cpu_one[0], "cores": 1,
                             "sample": f"{cpu_one[1]} oracle RK4 step(s) on a 16^3 block ({cpu_one[2]:.1f} s)"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": flat_bytes, "d2h_bytes_per_step": flat_bytes,
                "steps": e2e_steps, "overlap": "independent steps; uploads and downloads on a copy stream overlap "
                                              "the neighbouring steps' compute (two device states)"},
        "gpu_launches": f64["launches"],
        "clocks": f64["clocks"],
        "accuracy": {"fp64_ham_l2_after": float(f64["l2"][0]), "fp64_mom_l2_after": float(max(f64["l2"][1:4])),
                     "fp64_det_gt_minus_1_l2_after": float(f64["alg"][0]), "fp64_trace_At_l2_after": float(f64["alg"][1]),
                     "parity": "FP64 RHS within 1e-12 per-variable relative of the CPU oracle (tests)"},
        "forms": {
            "fp32_rhs": {"value": world * pts * args.steps / (f32["ms"] * 1e-3), "unit": UNIT,
                         "ms_per_step": f32["ms"] / args.steps, "stage_ms": f32["stage_ms"],
                         "timed_through": "bssn_rk4_step: one single-precision conversion per step, each stage "
                                          "writing the next stage's single-precision input",
                         "stage_ms_from": "the fused stage kernel timed on two further steps of per-stage calls "
                                          "(without the single-precision stores)",
                         "kernel": "k_stage32t<8,0> (tiled FP32-RHS stage: TMA-staged ghosted tiles)",
                         "achieved_tflops": achieved32 / 1e12, "frac_of_fp32_peak": achieved32 / peak32,
                         # algorithmic bytes of the stage kernel per point and stage, averaged over
                         # the four stages: FP32 stencil input 96, FP32 tables 88, FP64 W 8, y0 192,
                         # acc read 144 and written 144, ynext 192
                         "hbm": {"bytes_per_point_stage": mean_stage_bytes("fp32"),
                                 "achieved_gbs": mean_stage_bytes("fp32") * pts / (f32["stage_ms"] * 1e-3) / 1e9,
                                 "frac": (mean_stage_bytes("fp32") * pts / (f32["stage_ms"] * 1e-3) / 1e9 /
                                          MEASURED["hbm_gbs"])
                                 if MEASURED.get("hbm_gbs") else None,
                                 "traffic": TRAFFIC_F32["bytes_per_launch_128"]
                                 if TRAFFIC_F32["src_sha"] == kernel32_src_sha() and n == N else None},
                         "err_vs_fp64_max_rel_per_tensor": float(np.max(err32)),
                         "err_vs_fp64_per_var": [float(x) for x in err32],
                         "ham_l2_after": float(f32["l2"][0]), "det_gt_minus_1_l2_after": float(f32["alg"][0]),
                         "trace_At_l2_after": float(f32["alg"][1]), "gpu_launches": f32["launches"],
                         "steps": args.steps + args.warmup},
            **batched,
        },
        "fp_rates_measured": rates,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--grid", type=int, default=N, help="interior points per axis (profiling: smaller cases)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 192-patch batched workload")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-corrector form")
    ap.add_argument("--no-amr", action="store_true", help="skip the refined-hierarchy (Berger-Oliger) form")
    ap.add_argument("--no-cfd", action="store_true", help="skip the CFD (SOLA Navier-Stokes) benchmark form")
    ap.add_argument("--cfd-only", action="store_true", help="run only the CFD benchmark form and print its numbers")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched-patch forms (FP64 and FP32-RHS) and print their numbers")
    ap.add_argument("--learned-only", action="store_true",
                    help="run only the learned-corrector form and print its numbers")
    ap.add_argument("--amr-only", action="store_true",
                    help="run only the refined-hierarchy forms (FP64 and FP32-RHS) and print their numbers")
    ap.add_argument("--no-fp32-config", action="store_true",
                    help="skip the FP32-RHS 256^3 throughput and 96^3 100-step accuracy runs")
    ap.add_argument("--learned-pairs", type=int, default=2000,
                    help="training pairs for the learned form (20 per fine trajectory)")
    ap.add_argument("--learned-epochs", type=int, default=10)
    ap.add_argument("--corrector-only", action="store_true",
                    help="only the learned corrector's kernels (training steps and forward passes, 64^3): for ncu")
    ap.add_argument("--profile", action="store_true",
                    help="only the FP64 and FP32 timed loops (no probe, e2e, CPU leg): for ncu captures")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
