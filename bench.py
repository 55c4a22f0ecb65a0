"""Benchmark: NEP-ZBL velocity-Verlet MD throughput (atom-steps/s) on one GB300.

Workload (default): the 8,192,000-atom bcc W slab (160^3 cells, a = 3.165 A,
periodic in x, y, open in z with 30 A of vacuum each side, 300 K velocities
from seed 5), random-init NEP-ZBL model (seed 1), FP32 descriptors/network
with FP64 positions/integrator/energy/virial, NVE at dt = 1 fs.  One "step"
is one MD step: kick-drift, cell binning, neighbour lists, descriptors,
network, pair forces + ZBL + virial, kick, thermo -- all in the library's CUDA
kernels, replayed from captured CUDA graphs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle (the
only reference that exists for this method) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_08140_gb300 import inputs as I  # noqa: E402

METRIC = "atom-steps/s for NEP-ZBL MD at 1M-8M atoms (FP32 vs plain FP64 GPU path); HBM roofline %"
UNIT = "atom-steps/s"
WORKLOAD = ("8,192,000-atom bcc W slab (160x160x160 cells, a=3.165 A), periodic x,y, open z "
            "with 30 A vacuum each side, 300 K (seed 5), NVE dt=1 fs, random-init NEP-ZBL "
            "(seed 1: r_c 6/4 A, n_max 4/4, basis 8, l_max 4 + 4-body, 30 neurons, ZBL 1/2 A)")

# FP32 issue rate used as the ALU roofline: SMs (read from the device) x 128
# FP32 lanes x 2 flop per FMA x SM clock.
FP32_LANES = 128

# Algorithmic work of one force evaluation, per atom and per ordered pair.
# Counted from the arithmetic the method needs in this formulation (an FMA is
# 2 flop; sqrt, reciprocal, sincospi and tanh count 1 each):
#   per radial pair, descriptor pass: distance 8, Chebyshev basis T_0..T_8 ~20,
#     5 radial functions g_n = f_c (C_n + sum_k h_nk T_k) 5*(18+2) = 100   -> 128
#   per angular pair, descriptor pass: Chebyshev 20, g_n 100, unit vector 4,
#     24 harmonics ~60, A_nlm += g_n Y_lm 240                               -> 424
#   per atom: q (120 squares/adds -> 240), 4-body 5*~60 = 300, network
#     forward 30x30 FMA 1800 + 30 tanh + 60, backward 30x30 FMA 1800,
#     adjoint dU/dq -> (b_k, A-bar) ~ 400                                   -> 4630
#   per radial pair, force pass: distance/unit vector 12, Chebyshev with
#     derivatives 40, sum_k b_k T_k and b_k T'_k 36, force 10, virial 18,
#     fixed-point conversion/scatter bookkeeping 6                          -> 122
#   per angular pair, force pass: Chebyshev with derivatives 40,
#     g_n and g'_n 190, harmonics 60, G_lm and G'_lm 480, S 96,
#     gradient polynomial contraction ~200, assembly 12                     -> 1078
FLOP_ATOM = 4630
FLOP_PAIR_R = 128 + 122
FLOP_PAIR_A = 424 + 1078

# Measured DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per
# atom: of the two timed force kernels (k_nep_ang_tm + both k_radial_force
# launches) per evaluation, and of every kernel of one MD step, from a
# one-pass capture of the 8,192,000-atom slab itself; used for that workload
# (scaled by the atom count for others).  Set to None when the kernels change
# until they are captured again.  Source:
# profiles/dram_bytes_md_step_slab_8192000.md.
DRAM_FORCE_PER_ATOM = 534.2
DRAM_STEP_PER_ATOM = 1275.9
# Compulsory HBM bytes per atom-step of this design: every array a kernel of
# the step needs read or written once by that kernel (neighbour records that
# the caches serve are not counted):
#   kick-drift x, v r/w + F, species read 124; binning x read, cell/slot/
#   relative position write 48; scatter 12; cell finalize 48; neighbour
#   search own position and cell read, lists (58 x 4 B) and counts, radial
#   descriptor write 280; angular kernel counts, angular entries (14 x 4 B),
#   position, q, index read, radial record write, own force accumulator 176;
#   radial forces counts, list (58 x 4 B), own record read, force
#   accumulator 288; accumulator clear 24; forces gather 52; second kick 76.
BYTES_STEP_ALG = 124 + 48 + 12 + 48 + 280 + 176 + 288 + 24 + 52 + 76
# L1/L2 gather bytes of the two force kernels (not DRAM): per atom its own
# position and counts (25 B); per radial pair the list entry read twice (8 B)
# and the neighbour's 48-byte record.
GATHER_ATOM = 25
GATHER_PAIR = 56


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
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
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _slab_cut(nl):
    """The full-depth slab cut to nl x nl cells across (open z, periodic x, y)."""
    pos = I.bcc(nl, nl, 160)
    pos[:, 2] += 30.0
    L = nl * I.A_W
    box = np.array([L, L, 160 * I.A_W + 60.0])
    pbc = np.array([1, 1, 0], np.int32)
    vel = I.maxwell_boltzmann(np.random.default_rng(5), len(pos), 300.0)
    return pos, vel, box, pbc


_SINGLE_THREAD = """
import sys, time, json
sys.path.insert(0, {root!r})
from oracle import oracle as O
from paper_2305_08140_gb300 import inputs as I
s = I.c1()
m = I.nep_model(1)
p, v, F, _ = O.md(m, s.pos, s.vel, s.box, s.pbc, s.mass, 1.0, 1)
t0 = time.perf_counter()
O.md(m, p, v, s.box, s.pbc, s.mass, 1.0, {steps}, forces=F)
dt = time.perf_counter() - t0
print(json.dumps({{"value": s.n * {steps} / dt, "threads": O.num_threads(), "seconds": dt}}))
"""


def cpu_baseline_sample() -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    four velocity-Verlet steps of a laterally cut piece of the slab (the full
    160-cell depth and both free surfaces, 32 x 32 cells across, 327,680
    atoms) on every host thread it uses, and, in a child process limited to
    one thread, 20 steps of the 2,000-atom crystal."""
    import subprocess
    from oracle import oracle as O
    nl, steps = 32, 4
    pos, vel, box, pbc = _slab_cut(nl)
    model = I.nep_model(1)
    p, v, F, _ = O.md(model, pos, vel, box, pbc, I.MASS_W, 1.0, 0)    # initial forces
    t0 = time.perf_counter()
    O.md(model, p, v, box, pbc, I.MASS_W, 1.0, steps, forces=F)
    dt = time.perf_counter() - t0
    n = len(pos)
    single = None
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        root = os.path.dirname(os.path.abspath(__file__))
        out = subprocess.run([sys.executable, "-c", _SINGLE_THREAD.format(root=root, steps=20)],
                             env=env, capture_output=True, text=True, timeout=300)
        single = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:   # the single-thread figure is context only
        single = {"error": str(e)[:200]}
    return {"value": n * steps / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": (f"FP64 oracle, {steps} velocity-Verlet steps of a {nl}x{nl}x160-cell cut "
                       f"of the slab ({n} atoms, open z, periodic x,y) in {dt:.1f} s"),
            "single_thread": {"value": single.get("value"), "unit": UNIT,
                              "sample": "FP64 oracle, 20 steps of the 2,000-atom crystal "
                                        "(10^3 cells), OMP_NUM_THREADS=1",
                              **{k: v for k, v in single.items() if k != "value"}}}


def _time_md(N, nep, s, steps, warm, dev, d_max=0.0, chunk=25):
    """Atom-steps/s of `steps` graph-replayed MD steps (CUDA events)."""
    import torch
    types = torch.tensor(s.types, dtype=torch.int32, device=dev)
    st = N.MDState(N.to_device_soa(s.pos, dev), N.to_device_soa(s.vel, dev), s.box, s.pbc,
                   dt_max=1.0, d_max=d_max, types=types)
    nep.set_option(N.NEP_OPT_GRAPH_CHUNK, min(chunk, steps))
    nep.md(st, warm)
    nep.md(st, min(chunk, steps))
    if steps % chunk and steps > chunk:
        nep.md(st, steps % chunk)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    nep.md(st, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": s.n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "atoms": s.n, "sim_time_fs": st.time}


def other_configs(dev):
    """Throughput of the other benchmark workloads (same library, same kernels)."""
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    model = I.nep_model(1)
    out = {}
    # the slab with a 0.5 A Verlet skin: lists rebuilt only after an atom moved 0.25 A
    s = I.c5()
    nep = N.NEP(model, "fp32")
    nep.set_option(N.NEP_OPT_SKIN_MILLIANGSTROM, 500)
    r = _time_md(N, nep, s, 100, 3, dev)
    r["list_builds"] = nep.stats()["list_builds_skin"]
    r["note"] = ("Verlet skin 0.5 A (lists with r_c + 0.5 A, rebuilt after a 0.25 A "
                 "displacement; pairs within r_c compacted every step)")
    out["c5_8192000_fp32_skin_0.5A"] = r
    nep.close()
    # the start of a foil cascade on the slab: Nose-Hoover chain (300 K) on the 3 a0
    # shell at the x and y faces, a 100 keV PKA 10 A below the top surface along
    # (1, 3, -5), variable time step (0.01 A per step, dt <= 1 fs)
    s = I.c5()
    nep = N.NEP(model, "fp32")
    grp = torch.tensor(I.border_group(s), dtype=torch.uint8, device=dev)
    nep.set_thermostat(300.0, tau=100.0, chain=4, group=grp)
    types = torch.tensor(s.types, dtype=torch.int32, device=dev)
    st = N.MDState(N.to_device_soa(s.pos, dev), N.to_device_soa(s.vel, dev), s.box, s.pbc,
                   dt_max=1.0, d_max=0.01, types=types)
    top = float(s.pos[:, 2].max())
    atom = nep.pka(st, (0.5 * s.box[0], 0.5 * s.box[1], top - 10.0), 1.0e5, (1.0, 3.0, -5.0))
    nep.set_option(N.NEP_OPT_GRAPH_CHUNK, 25)
    nep.md(st, 3)
    nep.md(st, 25)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    nep.md(st, 100)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["c5_8192000_cascade_start_fp32"] = {
        "value": s.n * 100 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / 100, "steps": 100,
        "atoms": s.n, "sim_time_fs": st.time, "pka_atom": atom,
        "thermostatted_atoms": int(grp.sum().item()),
        "note": ("Nose-Hoover chain on the 3 a0 shell of the periodic faces, 100 keV PKA "
                 "along (1, 3, -5), variable dt (0.01 A per step)")}
    nep.close()
    del s, st
    # the same slab as a random 50/50 W-Mo solid solution with a two-species model
    # (pair coefficient tables, mixed-Z ZBL, two masses)
    s = I.alloy(I.c5(), [0.5, 0.5], seed=305)
    nep = N.NEP(I.nep_model(301, species=("W", "Mo")), "fp32")
    r = _time_md(N, nep, s, 100, 3, dev)
    r["note"] = "two species (W, Mo), random labels, same geometry and velocities as the slab"
    out["c5_8192000_WMo_fp32"] = r
    nep.close()
    del s
    # equiatomic W-Mo-Ta-Nb, 128,000 atoms, four species, 1,000 steps
    s = I.hea()
    nep = N.NEP(I.nep_model(401, species=("W", "Mo", "Ta", "Nb")), "fp32")
    out["hea_WMoTaNb_128000_fp32"] = _time_md(N, nep, s, 1000, 3, dev)
    nep.close()
    del s
    # 2,000-atom bcc W: plain FP64 as configured, and the FP32 path; 100 NVE steps
    s = I.c1()
    for prec in ("fp64", "fp32"):
        nep = N.NEP(model, prec)
        out[f"c1_2000_{prec}"] = _time_md(N, nep, s, 100, 3, dev)
        nep.close()
    # 128,000-atom bcc W at 1000 K: FP32 path (1,000 steps) vs plain FP64 path (100 steps)
    s = I.c2()
    nep = N.NEP(model, "fp32")
    out["c2_128000_fp32"] = _time_md(N, nep, s, 1000, 3, dev)
    nep.close()
    nep = N.NEP(model, "fp64")
    out["c2_128000_fp64"] = _time_md(N, nep, s, 100, 3, dev)
    nep.close()
    # 250,000 atoms with a dense clump, variable time step (0.01 A per step), 500 steps
    s = I.c3()
    nep = N.NEP(model, "fp32")
    out["c3_250000_fp32_variable_dt"] = _time_md(N, nep, s, 500, 3, dev, d_max=0.01)
    nep.close()
    # 512 small periodic boxes: one persistent launch of forward + energy/force loss +
    # parameter gradient (targets from the seed-101 model evaluated by the same library)
    structs = I.c4()
    b = N.Batch(structs, dev)
    tgt = N.NEP(I.nep_model(101), "fp32")
    Et, Ft = tgt.batch_forward(b)
    tgt.close()
    nep = N.NEP(model, "fp32")
    bt, per = nep.batch_autotune(b, Et, Ft)
    for _ in range(3):
        nep.batch_loss_grad(b, Et, Ft)
    torch.cuda.synchronize()
    reps = 20
    t0 = time.perf_counter()
    for _ in range(reps):
        L, g, E, F = nep.batch_loss_grad(b, Et, Ft)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    out["c4_512_configs_loss_grad_fp32"] = {
        "value": b.N / dt, "unit": "atom-gradients/s", "ms_per_step": dt * 1e3,
        "configs": b.S, "atoms": b.N, "loss": L,
        "autotune": {"threads": bt, "ctas_per_sm": per,
                     "table": nep.batch_autotune_table()[0], "unit": "ms per fused launch"},
        "note": "host-timed synchronous API call (forward + loss + gradient)"}
    # one SNES generation of the paper's training (population 50, Sec. III.A) over the
    # same 512 configurations: candidates, the NEP loss of all 50 in one launch, update
    n_pop = 50
    d = len(model.params)
    mu = torch.tensor(model.params, dtype=torch.float64, device=dev)
    sigma = torch.full((d,), 0.01, dtype=torch.float64, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    samples = torch.randn((n_pop, d), generator=g, dtype=torch.float64, device=dev)
    Wt = torch.zeros((b.S, 6), dtype=torch.float64, device=dev)
    tgt_W = N.NEP(I.nep_model(101), "fp32")
    _, _, W9 = tgt_W.batch_forward(b, virials=True)
    tgt_W.close()
    Wt[:] = W9.reshape(b.S, 9)[:, [0, 4, 8, 5, 6, 1]]
    for _ in range(2):
        N.snes_generation(nep, b, mu, sigma, samples, Et, Ft, Wt)
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        losses = N.snes_generation(nep, b, mu, sigma, samples, Et, Ft, Wt)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    out["c4_512_configs_snes_generation_pop50_fp32"] = {
        "value": n_pop * b.N / dt, "unit": "atom-evaluations/s", "ms_per_step": dt * 1e3,
        "population": n_pop, "configs": b.S, "atoms": b.N,
        "best_loss": float(losses[:, 0].min()),
        "note": ("host-timed synchronous API call: candidates mu + sigma s_k, lists, 50 x 512 "
                 "forward passes with energy/force/virial RMSE and L1/L2 terms, ranking and "
                 "update; samples drawn once on the device and reused")}
    nep.close()
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    nl = 12
    pos, vel, box, pbc = _slab_cut(nl)
    model = I.nep_model(1)
    p, v, F, _ = O.md(model, pos, vel, box, pbc, I.MASS_W, 1.0, max(args.warmup, 0))
    t0 = time.perf_counter()
    p, v, F, _ = O.md(model, p, v, box, pbc, I.MASS_W, 1.0, args.steps, forces=F)
    dt = time.perf_counter() - t0
    n = len(pos)
    value = n * args.steps / dt
    sample = (f"FP64 oracle velocity-Verlet on a {nl}x{nl}x160-cell cut of the slab "
              f"({n} atoms, open z, periodic x,y), {args.steps} steps")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def replica_throughput(ms_local, n_local, steps, dist=None, device="cpu"):
    """Whole-job throughput of replicas: the slowest rank's time (max over
    ranks) and the atoms of all ranks x steps / that time.  Returns (ms, value)."""
    import torch
    ms, units = float(ms_local), float(n_local)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), float(u.item())
    return ms, units * steps / (ms * 1e-3)


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2305_08140_gb300 import nepzbl as N

    s = I.c5(ncell=args.ncell)
    n = s.n
    model = I.nep_model(1)
    nep = N.NEP(model, "fp32")
    dev = torch.device("cuda", local)
    x = N.to_device_soa(s.pos, dev)
    v = N.to_device_soa(s.vel, dev)
    st = N.MDState(x, v, s.box, s.pbc, dt_max=1.0)
    stream = torch.cuda.current_stream()

    # autotune (neighbour-search tiling, steps per graph) on this state, outside
    # the timed region; the state is not advanced
    tune = None
    if not args.no_tune:
        tune = nep.md_autotune(st, reps=2)
    chunk = nep.stats()["graph_chunk"] if tune else 25
    nep.set_option(N.NEP_OPT_GRAPH_CHUNK, chunk)
    # warm-up (includes the first force evaluation and graph capture)
    nep.md(st, max(args.warmup, 1))
    torch.cuda.synchronize()
    nep.set_option(N.NEP_OPT_TIMING, 1)
    # capture every graph length the timed run uses outside the timed region
    nep.md(st, min(chunk, args.steps))
    if args.steps % chunk and args.steps > chunk:
        nep.md(st, args.steps % chunk)
    nep.reset_stats()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    nep.md(st, args.steps, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    stats = nep.stats()
    ms, value = replica_throughput(ms, n, args.steps, dist, dev)

    # roofline of the dominant kernel (the force kernel), timed inside the region
    peaks, peak_kind = _measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    k_ms = stats["timed_ms"] / max(stats["timed_launches"], 1)
    pr, pa = stats["pairs_radial"], stats["pairs_angular"]
    # when the neighbour-list kernel sums the radial descriptor, its 128 flop per
    # radial pair are done outside the timed force kernels and are not counted
    q_fused = bool(stats["radial_q_in_neighbor_kernel"])
    flop = FLOP_ATOM * n + (FLOP_PAIR_R - (128 if q_fused else 0)) * pr + FLOP_PAIR_A * pa
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    achieved = flop / (k_ms * 1e-3) / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # DRAM bytes of the timed kernels (ncu) over their live duration
    traffic = DRAM_FORCE_PER_ATOM * n if (q_fused and DRAM_FORCE_PER_ATOM) else None
    hbm_kernel = traffic / (k_ms * 1e-3) / 1e9 if traffic else None
    gather_gbs = (GATHER_ATOM * n + GATHER_PAIR * pr) / (k_ms * 1e-3) / 1e9
    launches = stats["kernel_launches"]

    # FP64 path on the same workload (a few steps)
    nep.set_option(N.NEP_OPT_TIMING, 0)
    fp64 = None
    if not args.skip_fp64:
        nep64 = N.NEP(model, "fp64")
        st64 = N.MDState(N.to_device_soa(s.pos, dev), N.to_device_soa(s.vel, dev), s.box, s.pbc,
                         dt_max=1.0)
        nep64.set_option(N.NEP_OPT_GRAPH_CHUNK, 2)
        nep64.md(st64, 1)
        torch.cuda.synchronize()
        k64 = 2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nep64.md(st64, k64, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"value": n * k64 / (e0.elapsed_time(e1) * 1e-3), "unit": UNIT, "steps": k64,
                "dtype": "f64"}
        nep64.close()
        del st64

    # end to end through the C ABI with host buffers (md_step_host): every step
    # copies x, v, F and the species from pinned host memory, runs one MD step
    # and copies x, v, F and the step's energies, virial and status back
    k_e2e = max(1, min(args.steps, 10))
    nep.set_option(N.NEP_OPT_TIMING, 0)
    hst = N.MDState(st.xyz.cpu().pin_memory(), st.vel.cpu().pin_memory(), s.box, s.pbc,
                    dt_max=1.0, types=st.types.cpu().pin_memory(),
                    forces=st.forces.cpu().pin_memory())
    nep.md_host(hst, 1, stream)        # device mirror allocated, 1-step graph captured
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        nep.md_host(hst, 1, stream)
        _ = hst.potential_energy
    e2e_s = time.perf_counter() - t0
    # per step: x, v, F (3 x 24 B) and species (4 B) per atom in plus the thermo
    # block (20 doubles); x, v, F out plus status, pair counts, energy/virial and
    # thermo (3 + 4 + 10 + 20 words)
    e2e = {"value": ws * n * k_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 76 * n + 160,
           "d2h_bytes_per_step": 72 * n + 268, "steps": k_e2e,
           "call": "md_step_host (C ABI, host arrays)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline_sample()
    others = None
    if rank == 0 and not args.skip_extras:
        del st
        torch.cuda.empty_cache()
        others = other_configs(dev)

    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded bcc W lattice, random-init NEP-ZBL weights)",
        "config": {"workload": WORKLOAD if args.ncell == 160 else
                   f"PROFILING CASE {args.ncell}^3-cell slab, {n} atoms", "atoms": n, "precision": "fp32 descriptors/network/forces,"
                   " fp64 positions/integrator/energy/virial", "parallelism": "replicas" if ws > 1
                   else "single GPU", "l2": "inputs larger than L2 (state ~0.6 GB, lists ~3 GB)",
                   "graph_chunk": chunk},
        "autotune": ({"tiling": {"kept": tune["tiling"][1], "table": tune["tiling"][0],
                                 "unit": "ms per force evaluation"},
                      "graph_chunk": {"kept": tune["graph_chunk"][1],
                                      "table": tune["graph_chunk"][0],
                                      "unit": "ms per MD step"}} if tune else None),
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": {"bound": "alu",
                     "kernel": ("k_nep_ang_tm + k_radial_force (angular descriptor, network, "
                                "forces, angular state in Tensor Memory; radial descriptor "
                                "summed in k_neighbors)" if q_fused
                                else "k_radial_q + k_nep_ang + k_radial_force"),
                     "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops,
                     "traffic": traffic,
                     "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                      "timed kernels per evaluation, one-pass capture of the "
                                      "8,192,000-atom slab (scaled by atoms for other sizes); "
                                      "null while the kernels differ from the capture"),
                     "peak_kind": f"FP32 issue rate {sms} SMs x {FP32_LANES} lanes x 2 x "
                                  f"{sm_mhz:.0f} MHz (sm_max_mhz, {peak_kind})",
                     "sm_count": sms,
                     "kernel_ms": k_ms, "flop_per_launch": flop,
                     "hbm_achieved_gbs": hbm_kernel, "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": hbm_kernel / hbm_peak if hbm_kernel else None,
                     "hbm_note": "measured DRAM bytes of the timed kernels / their live "
                                 "CUDA-event duration / measured copy bandwidth",
                     "l1l2_gather_gbs": gather_gbs,
                     "l1l2_gather_note": "bytes the force kernels gather through L1/L2 (own "
                                         "position and counts 25 B per atom, 56 B per radial "
                                         "pair), not DRAM",
                     "kernel_share": stats["timed_ms"] / ms if ms > 0 else None,
                     "pairs_radial": pr, "pairs_angular": pa,
                     # tiles of 128 atoms of the last graph chunk, and those that
                     # held a dense clump and ran in the register angular kernel (the
                     # rest kept their angular state in Tensor Memory)
                     "angular_tiles": stats["angular_tiles"],
                     "angular_tiles_register": stats["angular_tiles_register"]},
        "step_hbm": {
            "bytes_per_atom_step": BYTES_STEP_ALG,
            "achieved_gbs": BYTES_STEP_ALG * n * args.steps / (ms * 1e-3) / 1e9,
            "frac": BYTES_STEP_ALG * n * args.steps / (ms * 1e-3) / 1e9 / hbm_peak,
            "measured_bytes_per_atom_step": DRAM_STEP_PER_ATOM,
            "measured_gbs": (DRAM_STEP_PER_ATOM * n * args.steps / (ms * 1e-3) / 1e9
                             if DRAM_STEP_PER_ATOM else None),
            "measured_frac": (DRAM_STEP_PER_ATOM * n * args.steps / (ms * 1e-3) / 1e9 / hbm_peak
                              if DRAM_STEP_PER_ATOM else None),
            "note": "whole MD step: compulsory bytes of this design's kernels (and ncu DRAM "
                    "bytes of one step) x atoms / ms_per_step / measured copy bandwidth"},
        "fp64_path": fp64,
        "other_configs": others,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    return 0


def run_profile_case(args):
    """One workload, a few repetitions, no JSON line: the command that ncu
    captures for the kernels outside the MD step (one kernel per capture).
      c4_loss     512 configurations, fused forward + loss + gradient (k_batch)
      c4_pop      the NEP loss of a population of 50 over the 512 configurations
                  (k_batch_pop)
      c2_fp64     one plain-FP64 force evaluation of the 128,000-atom crystal
                  (k_nep_ang<double>, k_radial_force<double>)
      wmo_md      MD of the 8,192,000-atom slab as a 50/50 W-Mo alloy: 3 steps,
                  then graph chunks of 5 (the several-species kernels)
      c3_md       MD of the 250,000-atom crystal with a dense clump, variable dt
                  (0.01 A per step): 3 steps, then graph chunks of 5
    """
    import torch
    from paper_2305_08140_gb300 import nepzbl as N
    dev = torch.device("cuda", 0)
    model = I.nep_model(1)
    reps = max(args.steps, 1)
    if args.profile_case in ("c4_loss", "c4_pop"):
        structs = I.c4()
        b = N.Batch(structs, dev)
        tgt = N.NEP(I.nep_model(101), "fp32")
        Et, Ft, W9 = tgt.batch_forward(b, virials=True)
        tgt.close()
        nep = N.NEP(model, "fp32")
        if args.profile_case == "c4_loss":
            for _ in range(reps):
                nep.batch_loss_grad(b, Et, Ft)
        else:
            Wt = W9.reshape(b.S, 9)[:, [0, 4, 8, 5, 6, 1]].contiguous()
            g = torch.Generator(device=dev)
            g.manual_seed(7)
            theta = torch.tensor(model.params, dtype=torch.float64, device=dev)
            thetas = theta[None, :] + 0.01 * torch.randn((50, theta.numel()), generator=g,
                                                          dtype=torch.float64, device=dev)
            for _ in range(reps):
                N.population_loss(nep, b, thetas, Et, Ft, Wt)
        nep.close()
    elif args.profile_case == "c3_md":
        s = I.c3()
        nep = N.NEP(model, "fp32")
        st = N.MDState(N.to_device_soa(s.pos, dev), N.to_device_soa(s.vel, dev), s.box, s.pbc,
                       dt_max=1.0, d_max=0.01)
        nep.set_option(N.NEP_OPT_GRAPH_CHUNK, 5)
        nep.md(st, 3)
        for _ in range(reps):
            nep.md(st, 5)
        torch.cuda.synchronize()
        nep.close()
    elif args.profile_case == "wmo_md":
        s = I.alloy(I.c5(), [0.5, 0.5], seed=305)
        nep = N.NEP(I.nep_model(301, species=("W", "Mo")), "fp32")
        types = torch.tensor(s.types, dtype=torch.int32, device=dev)
        st = N.MDState(N.to_device_soa(s.pos, dev), N.to_device_soa(s.vel, dev), s.box, s.pbc,
                       dt_max=1.0, types=types)
        nep.set_option(N.NEP_OPT_GRAPH_CHUNK, 5)
        nep.md(st, 3)
        for _ in range(reps):
            nep.md(st, 5)
        torch.cuda.synchronize()
        nep.close()
    elif args.profile_case == "c2_fp64":
        s = I.displaced(I.c2(), 0.05, 41)
        nep = N.NEP(model, "fp64")
        x = N.to_device_soa(s.pos, dev)
        for _ in range(reps):
            nep.compute(x, s.box, s.pbc)
        nep.close()
    torch.cuda.synchronize()
    print(f"profile case {args.profile_case}: {reps} repetitions done")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the measurements of the other workloads")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the MD autotuner (default options: 1 z slice, chunk 16, 25 steps "
                         "per graph)")
    ap.add_argument("--ncell", type=int, default=160,
                    help="slab size in bcc cells per side (160 = the 8,192,000-atom workload; "
                         "smaller values only for profiling)")
    ap.add_argument("--profile-case", choices=["c4_loss", "c4_pop", "c2_fp64", "wmo_md", "c3_md"], default=None,
                    help="run one other workload --steps times without timing (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
