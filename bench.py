"""Benchmark of the LRDMC hot path on one B300 (or N independent replicas).

One *step* is one branching interval of the load-balanced schedule over the
whole population: N_proj = 20 lattice hops for every walker (evaluation of all
6 N_e hop ratios, diagonal W and local energy, weight update, heat-bath hop,
Sherman-Morrison update) followed by the branching step (statistics,
integer-comb reconfiguration, gather).  Workload: the synthetic water-methane
complex (16 valence electrons, 56 Gaussian basis functions, 8 nuclei), 4096
walkers, a = 0.2 bohr, FP64.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm of this benchmark) on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_W = 4096
N_PROJ = 20
A = 0.2
SEED = 1
FP64_PEAK_GFLOPS = 1250.0      # nominal B300 FP64 rate (profiling recipe table)
# FP64 rate from unit counts: 148 SMs x 2 FP64 FMA lanes per clock (the peak
# ncu reports for the FP64 pipe) x 2 FLOP x 2.032 GHz maximum SM clock
FP64_UNIT_COUNT_GFLOPS = 148 * 2 * 2 * 2.032
# DRAM bytes (read + write) of one k_propagate launch of this workload, the
# FP64 pipe busy fraction, and the FP64 warp instructions per walker-step with
# their mean active lanes (sm__inst_executed_pipe_fp64,
# sm__thread_inst_executed_pipe_fp64_pred_on), from one ncu capture of the
# propagate kernel (second launch of `bench.py --steps 2 --warmup 1` with every
# extra section off); None when the kernel has changed since that capture
PROPAGATE_TRAFFIC_BYTES = 1.204502784e9 + 0.671022336e9
PROPAGATE_FP64_PIPE_BUSY = 0.8270
PROPAGATE_FP64_INST_PER_STEP = 51511632 / 81920
PROPAGATE_FP64_ACTIVE_LANES = 1384697504 / 51511632
# walkers per host process in the oracle sample (cpu_baseline and the
# reference arm): one warm-up interval, then one timed 20-hop interval
ORACLE_WALKERS_PER_PROC = 8
# FP64 pipe instructions of the functions as the propagate kernel implements
# them: table-driven exp (10), approximate reciprocal / rsqrt plus one
# third-order refinement (4 / 6), tabulated erf(r/r_c)/r (index 3, Horner 10,
# scalings 2).
OP_EXP, OP_RSQ, OP_RCP, OP_ERF = 9.0, 6.0, 4.0, 15.0
OP_PADE_VALUE = OP_RSQ + 1 + OP_RCP + 1          # u = c / (1/r + b)
OP_PADE = OP_RSQ + 1 + OP_RCP + 1 + 1 + 2 + 3    # u, u', u'' and 1/r


def json_line(obj) -> str:
    """The result line as strict JSON: a value that is not finite (an error bar
    over too few intervals) is written as null."""
    def clean(v):
        if isinstance(v, dict):
            return {k: clean(x) for k, x in v.items()}
        if isinstance(v, (list, tuple)):
            return [clean(x) for x in v]
        if isinstance(v, (float, np.floating)):
            return float(v) if math.isfinite(v) else None
        if isinstance(v, np.integer):
            return int(v)
        return v
    return json.dumps(clean(obj), allow_nan=False)


def algorithmic_ops_per_walker_step(n_e, n_nuc, n_bf, n_prim, n_sig, n_s_shell, n_p_shell):
    """FP64 operations per walker-step of the load-balanced step as formulated
    in the propagate kernel (one add/mul/FMA = 1; a function counts its FP64
    instructions above).  Every walker-step is one hop of an electron m and the
    incremental evaluation that follows it; the caches persist across
    branching intervals, so no step pays a full evaluation.

    Move: basis value/gradient/Laplacian at the new position (per primitive an
    exponential + 10), the 5 n_sig x n_bf contraction, Sherman-Morrison
    (2 n_sig^2) and the n_sig x n_bf update of g, the potentials (per nucleus
    erf + 8; the 1/r is shared with m's one-body Jastrow term).  Evaluation:
    m's pair and nucleus terms with derivatives
    and the partner electrons' swapped terms (Pade + 14 per partner, 14 per
    swap), determinant derivatives of m's block (4 n_sig^2), basis values at
    m's six hops (below) and their Jastrow terms (Pade value + 3 per partner), the block's hop
    determinant ratios from cached basis values (6 n_sig n_bf), the swapped
    pair terms of the other hops (2 each), every hop's exponential (+3) and the
    assembly (20 per electron).  The basis values at m's six hops factor per
    Gaussian primitive into exp(-z (d^2 + a^2)) and, per hop axis,
    exp(-2 z a |d_k|) and its reciprocal (4 exponentials, 3 reciprocals and
    18 other operations per primitive), plus the 18 Cartesian factors
    (2 operations each) of every p shell."""
    del n_s_shell
    per = n_e - 1 + n_nuc
    move = (n_prim * (OP_EXP + 10) + 5 * n_bf * n_sig + 2 * n_sig * n_sig + n_sig * n_bf
            + n_nuc * (OP_ERF + 8))
    hop_basis = n_prim * (OP_EXP + 3 + 3 * (OP_EXP + OP_RCP + 5)) + 18 * 2 * n_p_shell
    evaluation = (per * (OP_PADE + 14) + (n_e - 1) * 14 + 4 * n_sig * n_sig
                  + hop_basis + 6 * per * (OP_PADE_VALUE + 3)
                  + 6 * n_sig * n_bf + 6 * (n_e - 1) * 2 + 6 * n_e * (OP_EXP + 3) + 20 * n_e)
    return move + evaluation


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and clock-event reasons during a timed region: NVML every 5 ms
    from a thread (the GPU found by the CUDA device's PCI bus id), else
    nvidia-smi every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.nvml = None
        self.stop = threading.Event()
        self.source = None

    def _nvml_handle(self):
        """NVML through the driver's libnvidia-ml (public C API, read-only calls)."""
        import ctypes
        import torch
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        pr = torch.cuda.get_device_properties(self.gpu)
        h = ctypes.c_void_p()
        bus = b"%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        if nv.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
            raise OSError("no NVML device at " + bus.decode())
        return nv, h

    def __enter__(self):
        try:
            nv, h = self._nvml_handle()
            self.nvml = (nv, h)
            self.source = "nvml"
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _poll(self):
        import ctypes
        nv, h = self.nvml
        NVML_CLOCK_SM = 1
        clk, mx, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if nv.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx)) != 0:
            return
        while not self.stop.is_set():
            if (nv.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(clk)) != 0 or
                    nv.nvmlDeviceGetCurrentClocksThrottleReasons(h, ctypes.byref(bits)) != 0):
                break
            self.rows.append((float(clk.value), float(mx.value),
                              [nm for nm, b in self.REASONS if bits.value & b]))
            self.stop.wait(0.005)

    def _read(self):
        names = [nm for nm, _ in self.REASONS]
        for line in self.proc.stdout:
            r = [v.strip() for v in line.split(",")]
            if len(r) >= 9 and r[1].replace(".", "").isdigit() and r[2].replace(".", "").isdigit():
                self.rows.append((float(r[1]), float(r[2]),
                                  [nm for k, nm in enumerate(names) if r[5 + k].lower().startswith("active")]))

    def __exit__(self, *a):
        self.stop.set()
        if self.nvml:
            self.t.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [r[0] for r in self.rows]
        mx = [r[1] for r in self.rows]
        reasons = sorted({nm for r in self.rows for nm in r[2]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm), "source": self.source}


# ----------------------------------------------------------------- oracle baseline
def _oracle_chunk(args):
    """One host process's share of the oracle sample: its walkers are set up
    and run one load-balanced warm-up interval untimed, then one timed
    20-hop interval (steady state, as the GPU's timed intervals are)."""
    ids, n_proj = args
    import workloads as W
    from oracle import lrdmc as L
    s = W.water_methane()
    x = W.initial_walkers(s, N_W, seed=SEED + 10)[ids]
    Wk = L.init_walkers(s, x, A)
    E0 = float(np.mean(Wk.ev["eL"]))
    L.propagate_lb(s, Wk, A, E0, n_proj, SEED, 0, walker_ids=ids)
    t = time.perf_counter()
    L.propagate_lb(s, Wk, A, E0, n_proj, SEED, 1, walker_ids=ids)
    return time.perf_counter() - t, len(ids) * n_proj


class OracleSample:
    """The CPU oracle timed on all host cores: one spawned process per core,
    each on its own ORACLE_WALKERS_PER_PROC walker slots of the benchmark
    population.  One sample = one timed 20-hop interval of every process
    (after its untimed set-up and warm-up interval); its time is the slowest
    process's interval and its rate the walker-steps of all processes over
    that time."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def describe(self):
        return (f"{self.procs} processes x {ORACLE_WALKERS_PER_PROC} walkers, one timed {N_PROJ}-hop "
                f"load-balanced interval each after one untimed warm-up interval "
                f"({self.procs * ORACLE_WALKERS_PER_PROC * N_PROJ} walker-steps per sample)")

    def run(self, k=0):
        n = ORACLE_WALKERS_PER_PROC
        jobs = [((np.arange(n) + (j * n + k * self.procs * n)) % N_W, N_PROJ) for j in range(self.procs)]
        res = self.pool.map(_oracle_chunk, jobs)
        steps = sum(r[1] for r in res)
        slowest = max(r[0] for r in res)
        return steps / slowest, slowest, steps

    def close(self):
        self.pool.close()
        self.pool.join()


def measure_fp64_peak(dev_index=0):
    """FP64 FMA peak of this GPU from bench_fp64_peak.cu (built here with nvcc
    into _build/, run under the clock sampler); None if it cannot be built."""
    src = os.path.join(ROOT, "bench_fp64_peak.cu")
    out_dir = os.path.join(ROOT, "_build")
    exe = os.path.join(out_dir, "bench_fp64_peak")
    try:
        if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
            os.makedirs(out_dir, exist_ok=True)
            from paper_2508_12033_b300.build import nvcc_path, ARCH
            subprocess.run([nvcc_path(), "-O3", "-gencode", ARCH, "-o", exe + ".tmp", src], check=True,
                           capture_output=True)
            os.replace(exe + ".tmp", exe)
        env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", str(dev_index)))
        with ClockSampler(dev_index) as clk:
            r = subprocess.run([exe], check=True, capture_output=True, text=True, env=env, timeout=120)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        d["clocks"] = clk.summary()
        return d
    except Exception as e:      # noqa: BLE001 (reported in the JSON line)
        return {"error": f"{type(e).__name__}: {e}"[:200]}


# ----------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import torch
    import workloads as W
    from paper_2508_12033_b300 import build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()                   # the other ranks load the library rank 0 made current
    import paper_2508_12033_b300 as P

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    s = W.water_methane()
    x0 = W.initial_walkers(s, N_W, seed=SEED + 10 + rank)
    lr = P.Lrdmc(s, x0, A, seed=SEED + rank, reinv_period=100, p_gbar=10)
    stream = lr.stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 126 MB L2

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        lr.propagate(P.LOAD_BALANCED, n_proj=N_PROJ)
        lr.branch()
    torch.cuda.synchronize()
    barrier()
    n0 = lr.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        barrier()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)               # L2 flush between timed steps (not timed)
                ev[k][0].record(stream)
                lr.propagate(P.LOAD_BALANCED, n_proj=N_PROJ)
                ev[k][1].record(stream)
                lr.branch()                          # synchronises on its statistics readback
                ev[k][2].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = lr.launch_count() - n0
    step_ms = [e0.elapsed_time(e2) for e0, _, e2 in ev]
    prop_ms = [e0.elapsed_time(e1) for e0, e1, _ in ev]
    ws_per_step = N_W * N_PROJ
    value, t_total = aggregate_throughput(sum(step_ms) / 1e3, ws_per_step * args.steps, world, dev)
    # roofline of the dominant kernel (the propagate kernel: one launch per step)
    slots = algorithmic_ops_per_walker_step(s.n_elec, s.n_nuc, s.n_bf, s.n_prim_eval, max(s.n_up, s.n_dn),
                                            int(np.sum(s.shell_l == 0)), int(np.sum(s.shell_l == 1)))
    prop_s = statistics.mean(prop_ms) / 1e3
    achieved = 2.0 * slots * ws_per_step / prop_s / 1e9      # GFLOP/s, FP64-equivalent
    # conventional schedule at the same mean hops per interval (tau = N_proj / <b_bar>)
    g = lr.get_walkers()
    tau = N_PROJ / float(np.mean(g["ev"][:, 0]))
    conv_ms, conv_moves = [], []
    for k in range(max(2, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lr.propagate(P.CONVENTIONAL, tau=tau, max_moves=100 * N_PROJ)
            lr.branch()
            e1.record(stream)
        torch.cuda.synchronize()
        conv_ms.append(e0.elapsed_time(e1))
        h = lr.history()
        conv_moves.append((float(h["moves_mean"][-1]), int(h["moves_max"][-1])))
    conv_rate = N_W * statistics.mean(m for m, _ in conv_moves) / (statistics.mean(conv_ms) / 1e3)
    # load imbalance inside the GPU: per-walker start/stop stamps of one interval
    lr.set_timing(True)
    imbalance = {}
    for name, kind in (("load_balanced", P.LOAD_BALANCED), ("conventional", P.CONVENTIONAL)):
        lr.propagate(kind, n_proj=N_PROJ, tau=tau, max_moves=100 * N_PROJ)
        imbalance[name] = lr.interval_timing()
        lr.branch()
    lr.set_timing(False)
    # end to end through the public API with host buffers: upload the walkers
    # from pinned host memory (re-initialising them), one interval + branching,
    # read back the population (positions, weights, b_bar / V_sf / W / e_L,
    # status, moves) into pinned host memory
    def pinned(shape, dt):
        return torch.empty(shape, dtype=dt).pin_memory().numpy()
    ne = s.n_elec
    host = dict(x=pinned((N_W, ne, 3), torch.float64), w=pinned((N_W,), torch.float64),
                ev=pinned((N_W, 4), torch.float64), status=pinned((N_W,), torch.int32).view(np.uint32),
                moves=pinned((N_W,), torch.int32))
    xh = pinned((N_W, ne, 3), torch.float64)
    xh[:] = lr.get_walkers(("x",))["x"]
    fields = tuple(host)
    e2e_ms = []
    for k in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lr.set_walkers(xh)
        lr.propagate(P.LOAD_BALANCED, n_proj=N_PROJ)
        lr.branch()
        lr.get_walkers(fields, out=host)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        xh[:] = host["x"]
    h2d = xh.nbytes
    d2h = sum(a.nbytes for a in host.values())
    e2e_value = world * ws_per_step / (statistics.mean(e2e_ms) / 1e3)
    mixed = run_mixed(args, P, s, x0, lr, flush, rank) if not args.no_mixed else None
    a_scan = run_a_scan(P) if rank == 0 and not args.no_a_scan else None
    h2 = run_h2(P) if rank == 0 and not args.no_a_scan else None
    adjoint = run_adjoint(P) if rank == 0 and not args.no_adjoint else None
    large = run_large(P, flush) if rank == 0 and not args.no_large else None
    batch = None
    if rank == 0 and not args.no_batch:
        batch = {"mixed": run_batch(P, 1), "fp64": run_batch(P, 0)}
    return dict(value=value, t_total=t_total, step_ms=statistics.mean(step_ms), prop_ms=statistics.mean(prop_ms),
                launches=launches, achieved=achieved, clocks=clk.summary(), conv_rate=conv_rate,
                conv_moves=conv_moves, tau=tau, e2e=e2e_value, h2d=h2d, d2h=d2h, slots=slots,
                energy=lr.energy(), mixed=mixed, imbalance=imbalance, a_scan=a_scan, h2=h2, batch=batch, adjoint=adjoint,
                large=large)


def aggregate_throughput(t_local, units_local, world, device="cpu"):
    """Whole-job throughput of independent replicas: total work of all ranks
    divided by the slowest rank's time (MAX over ranks, SUM of units)."""
    if world <= 1:
        return units_local / t_local, t_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def time_lb_intervals(lr, P, flush, steps, warmup):
    """Mean ms per load-balanced interval (propagate + branch), L2 flushed between."""
    import torch
    for _ in range(warmup):
        lr.propagate(P.LOAD_BALANCED, n_proj=N_PROJ)
        lr.branch()
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        with torch.cuda.stream(lr.stream):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(lr.stream)
            lr.propagate(P.LOAD_BALANCED, n_proj=N_PROJ)
            lr.branch()
            e1.record(lr.stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms)


def run_a_scan(P):
    """Lattice-space extrapolation: load-balanced LRDMC of the hydrogen atom
    (Slater guiding function exp(-0.8 r), walkers on the lattice a (Z^3 + 1/2))
    at four spacings, fitted to E_0 + c_2 a^2 + c_4 a^4; the continuum value is
    -1/2 Ha.  Reports the energies, the fit and the wall time of the scan."""
    import torch
    import workloads as W
    s = W.hydrogen_atom_sto(0.8)
    a_list, E_list, err_list = [0.3, 0.4, 0.5, 0.6], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a in a_list:
        lr = P.Lrdmc(s, W.lattice_walkers(2048, a, seed=4, spread=3), a, seed=11, p_gbar=20, n_equil=20)
        for _ in range(140):
            lr.propagate(P.LOAD_BALANCED, n_proj=15)
            lr.branch()
        E, err = lr.energy()
        E_list.append(E)
        err_list.append(err)
        del lr
    wall = time.perf_counter() - t0
    coef, cov, chi2 = P.extrapolate_a(a_list, E_list, err_list, 2)
    return {"system": "H atom, Slater guide exp(-0.8 r), 2048 walkers, 140 intervals x 15 hops per spacing",
            "a": a_list, "E": E_list, "err": err_list, "E0": float(coef[0]), "E0_err": float(np.sqrt(cov[0, 0])),
            "chi2": chi2, "exact_continuum": -0.5, "wall_s": wall}


def run_h2(P):
    """The H2 run at its stated size: STO-3G H2 (2 electrons, nuclei at
    z = +-0.7 bohr), a = 0.2, 256 walkers, 100 branching intervals of 20
    moves (2000 steps), Philox seed 1, node rule 2 (the cap on every electron:
    the cusp-less Gaussian orbital leaves W unbounded below otherwise), both
    schedules; the conventional projection time gives the same mean move
    count (tau = 20 / <b_bar>, b_bar averaged over the walkers at the end of the
    load-balanced run's first five intervals).  Absolute
    numbers only: the 256 walkers (3072 hop evaluations per step) leave the
    GPU mostly idle."""
    import torch
    import workloads as W
    s = W.h2_sto3g()
    x0 = W.initial_walkers(s, 256, seed=11)
    out = {"system": "H2 STO-3G, a = 0.2, 256 walkers, 100 intervals x 20 moves, node rule 2"}
    tau, bbar = None, []
    for kind, name in ((P.LOAD_BALANCED, "load_balanced"), (P.CONVENTIONAL, "conventional")):
        lr = P.Lrdmc(s, x0, 0.2, seed=1, p_gbar=10, n_equil=10, node_rule=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(100):
            lr.propagate(kind, n_proj=20, tau=tau or 0.0, max_moves=100000)
            if kind == P.LOAD_BALANCED and j < 5:      # mean b_bar of the first five intervals' walkers
                bbar.append(float(np.mean(lr.get_walkers(("ev",))["ev"][:, 0])))
            lr.branch()
        if kind == P.LOAD_BALANCED:
            tau = 20.0 / float(np.mean(bbar))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        E, err = lr.energy()
        h = lr.history()
        moves = float(np.sum(h["moves_mean"])) * 256
        out[name] = {"E": E, "err": err, "wall_s": wall, "walker_steps_per_s": moves / wall,
                     "moves_mean": float(np.mean(h["moves_mean"])), "status_or": int(np.bitwise_or.reduce(h["status_or"]))}
        lr.close()
    out["tau"] = tau
    # lattice extrapolation of the same molecule (nodeless guiding function:
    # fixed node is exact, E(a -> 0) = -1.17447 Ha, the exact H2 energy at
    # R = 1.4 bohr); spacings below 0.15, where the bias of the cusp-less
    # Gaussian orbital follows a^2 + a^4
    spacings, Es, errs = [0.05, 0.07, 0.1, 0.14], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a in spacings:
        n_proj = int(round(20 * (0.2 / a) ** 2))
        lr = P.Lrdmc(s, W.initial_walkers(s, 4096, seed=5), a, seed=7, p_gbar=10, n_equil=75, node_rule=2)
        for _ in range(300):
            lr.propagate(P.LOAD_BALANCED, n_proj=n_proj)
            lr.branch()
        E, err = lr.energy()
        Es.append(E)
        errs.append(err)
        lr.close()
    coef, cov, chi2 = P.extrapolate_a(spacings, Es, errs, 2)
    out["a_scan"] = {"a": spacings, "E": Es, "err": errs, "walkers": 4096, "intervals": 300,
                     "moves_per_interval": "20 (0.2/a)^2", "E0": float(coef[0]), "E0_err": float(np.sqrt(cov[0, 0])),
                     "chi2": chi2, "exact": -1.17447, "wall_s": time.perf_counter() - t0}
    return out


def run_adjoint(P):
    """Hand-written adjoint: e_L, log|Psi| and their gradients with respect to
    all 384 nuclear coordinates and the 259 Jastrow parameters of the H128 chain
    (spacing 1.8 bohr, s + p GTO per atom, seeded MOs, a = 0.25) at 8192 seeded
    configurations, evaluated in one launch."""
    import torch
    import workloads as W
    s = W.hydrogen_chain(128)
    lr = P.Lrdmc(s, W.initial_walkers(s, 1024, seed=5), 0.25)
    x = torch.tensor(W.initial_walkers(s, 8192, seed=6), device="cuda")
    lr.local_energy_grad(x[:1024].contiguous())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eL, lp, ge, gl = lr.local_energy_grad(x)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    finite = bool(torch.isfinite(eL).all() and torch.isfinite(ge).all() and torch.isfinite(gl).all())
    return {"system": "H128 chain, 8192 configurations, FP64", "parameters": lr.param_count(),
            "ms": dt * 1e3, "configurations_per_s": 8192 / dt,
            "gradient_components_per_s": 2 * 8192 * lr.param_count() / dt, "all_finite": finite}


def run_large(P, flush, steps=3):
    """Single large systems: hydrogen clusters of 64 and 128 atoms (all-electron,
    s + p GTO per atom) at a = 0.25, load-balanced intervals of 20 hops, FP64 and
    mixed.  Their shared-memory layouts would leave fewer than 8 warps per SM,
    so both kernels run with the working sets in global memory."""
    import workloads as W
    out = {}
    for n_atoms, n_w in ((64, 4096), (128, 1024)):
        s = W.hydrogen_cluster(n_atoms, seed=3)
        x0 = W.initial_walkers(s, n_w, seed=11)
        for prec, name in ((0, "fp64"), (1, "mixed")):
            lr = P.Lrdmc(s, x0, 0.25, seed=SEED, reinv_period=50, p_gbar=10, precision=prec)
            ms = time_lb_intervals(lr, P, flush, steps, 2)
            lr.close()
            out[f"H{n_atoms}_{name}"] = {"n_e": s.n_elec, "n_w": n_w, "ms_per_step": ms,
                                         "value": n_w * N_PROJ / (ms / 1e3), "unit": "walker-steps/s"}
    return out


def run_batch(P, precision, steps=3):
    """Batched multi-system propagation: 64 seeded hydrogen clusters with N_e
    uniform in 16..128, 256 walkers each, a = 0.25, one persistent launch per
    interval.
    Walker-steps/s of load-balanced intervals (N_proj = 20) with each item order,
    the autotuned launch shape, and the SM idle time of a load-balanced and a
    conventional interval of equal mean hop count (the in-GPU image of the
    paper's weak-scaling loss)."""
    import torch
    import workloads as W
    rng = np.random.default_rng(3)
    ne = [int(v) for v in rng.integers(16, 129, size=64)]
    systems = [W.hydrogen_cluster(n, seed=100 + k) for k, n in enumerate(ne)]
    x0s = [W.initial_walkers(s, 256, seed=k) for k, s in enumerate(systems)]
    b = P.LrdmcBatch(systems, x0s, 0.25, list(range(1, 65)), reinv_period=50, precision=precision)
    best, tune_ms = b.tune(P.LOAD_BALANCED, n_proj=20)
    b.set_timing(True)
    out = {"systems": 64, "n_e": [min(ne), max(ne)], "walkers": 64 * 256, "precision": precision,
           "tuned_ctas_per_sm": best, "tune_ms": tune_ms}
    walker_steps = 64 * 256 * 20
    for pol in (1, 0):
        b.set_order(pol)
        b.propagate(P.LOAD_BALANCED, n_proj=20)
        b.branch()
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.propagate(P.LOAD_BALANCED, n_proj=20)
            b.branch()
            e1.record(b.stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = b.timing()
        key = "cost_order" if pol == 1 else "system_order"
        out[key] = {"value": walker_steps / (statistics.mean(ms) / 1e3), "unit": "walker-steps/s",
                    "ms_per_step": statistics.mean(ms), "lb_timing": t}
    # conventional interval with the same mean hop count per walker
    b.set_order(1)
    bbar = [float(np.mean(h.get_walkers()["ev"][:, 0])) for h in b.handles]
    tau = 20.0 / float(np.mean(bbar))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.propagate(P.CONVENTIONAL, tau=tau, max_moves=2000)
    e1.record(b.stream)
    torch.cuda.synchronize()
    t = b.timing()
    mv = np.concatenate([h.get_walkers()["moves"] for h in b.handles])
    out["conventional"] = {"tau": tau, "ms": e0.elapsed_time(e1), "moves_mean": float(mv.mean()),
                           "moves_max": int(mv.max()), "timing": t}
    b.branch()
    b.close()
    return out


def run_mixed(args, P, s, x0, lr64, flush, rank):
    """Mixed-precision form: throughput at the benchmark size and at 51200
    walkers, and its energy bias against FP64 by correlated sampling on the
    equilibrated FP64 population (same configurations evaluated both ways,
    weighted as in the load-balanced estimator, w / (W - E_0) with w = 1)."""
    import torch
    import workloads as W
    lm = P.Lrdmc(s, x0, A, seed=SEED + rank, reinv_period=50, p_gbar=10, precision=1)
    ms = time_lb_intervals(lm, P, flush, args.steps, args.warmup)
    x = torch.tensor(lr64.get_walkers()["x"], device=flush.device)
    _, ev64, _ = lr64.eval_configs(x)
    _, ev32, _ = lm.eval_configs(x)
    torch.cuda.synchronize()
    ev64, ev32 = ev64.cpu().numpy(), ev32.cpu().numpy()
    f = 1.0 / (ev64[:, 2] - lr64.e0)
    d = ev32[:, 3] - ev64[:, 3]
    bias = float(np.sum(f * d) / np.sum(f))
    err = float(np.std(d) * np.sqrt(np.sum(f * f)) / np.sum(f))
    lm.close()
    big = 51200
    xb = W.initial_walkers(s, big, seed=SEED + 20 + rank)
    lb = P.Lrdmc(s, xb, A, seed=SEED + rank, reinv_period=50, p_gbar=10, precision=1)
    ms_big = time_lb_intervals(lb, P, flush, max(2, args.steps // 3), 2)
    lb.close()
    # the FP64 form at the same size, the reference of the speed-up at 51200 walkers
    lf = P.Lrdmc(s, xb, A, seed=SEED + rank, reinv_period=100, p_gbar=10)
    ms_big64 = time_lb_intervals(lf, P, flush, max(2, args.steps // 3), 2)
    lf.close()
    # the FP32 orbital contractions on the tensor cores: TF32, BF16 and split
    # TF32 (precision 2, 3, 4), speed at both sizes and the same correlated bias
    tc = {}
    for prec, name in ((2, "tf32"), (3, "bf16"), (4, "split_tf32")):
        lt = P.Lrdmc(s, x0, A, seed=SEED + rank, reinv_period=50, p_gbar=10, precision=prec)
        ms_t = time_lb_intervals(lt, P, flush, max(2, args.steps // 2), 2)
        _, evt, _ = lt.eval_configs(x)
        torch.cuda.synchronize()
        dt = evt.cpu().numpy()[:, 3] - ev64[:, 3]
        lt.close()
        lt = P.Lrdmc(s, xb, A, seed=SEED + rank, reinv_period=50, p_gbar=10, precision=prec)
        ms_tb = time_lb_intervals(lt, P, flush, max(2, args.steps // 3), 2)
        lt.close()
        tc[name] = {"precision": prec, "value_4096": N_W * N_PROJ / (ms_t / 1e3),
                    "value_51200": big * N_PROJ / (ms_tb / 1e3), "speedup_vs_fp64_51200": ms_big64 / ms_tb,
                    "speedup_vs_mixed_fp32_51200": ms_big / ms_tb,
                    "energy_bias_mHa": 1e3 * float(np.sum(f * dt) / np.sum(f)),
                    "energy_bias_err_mHa": 1e3 * float(np.std(dt) * np.sqrt(np.sum(f * f)) / np.sum(f)),
                    "max_abs_eL_diff_Ha": float(np.max(np.abs(dt)))}
    return {"value": N_W * N_PROJ / (ms / 1e3), "unit": "walker-steps/s", "ms_per_step": ms,
            "n_w_51200": {"value": big * N_PROJ / (ms_big / 1e3), "ms_per_step": ms_big,
                          "fp64_value": big * N_PROJ / (ms_big64 / 1e3), "fp64_ms_per_step": ms_big64,
                          "speedup_vs_fp64": ms_big64 / ms_big},
            "energy_bias_mHa": 1e3 * bias, "energy_bias_err_mHa": 1e3 * err,
            "bias_sample": f"{N_W} equilibrated FP64 configurations, weights 1/(W - E0)",
            "max_abs_eL_diff_Ha": float(np.max(np.abs(d))),
            "precision": "FP32 hop ratios / basis / Jastrow; FP64 A rows, B, Sherman-Morrison, accumulators",
            "tensor_core": tc}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrdmc", choices=["lrdmc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-a-scan", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    workload = {"workload": "water-methane complex: 8 nuclei (C, 4 H, O, 2 H), 16 valence electrons "
                            "(8 up, 8 down), erf-screened local pseudopotentials, 56 single-primitive GTOs, "
                            "seeded orthonormal MOs, Pade 1- and 2-body Jastrow; a = 0.2 bohr",
                "n_w": N_W, "n_e": 16, "n_proj": N_PROJ, "schedule": "load-balanced",
                "step": "one branching interval (20 hops per walker) + reconfiguration",
                "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{args.gpus}"}
    metric = "walker-steps/s (LRDMC load-balanced, FP64)"
    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        orc = OracleSample()
        rates, times = [], []
        for k in range(args.warmup + args.steps):
            r, slowest, steps = orc.run(k)
            if k >= args.warmup:
                rates.append(r)
                times.append(slowest)
        orc.close()
        v = statistics.mean(rates)
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "walker-steps/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload,
                "step": "one oracle sample (not the GPU arm's 4096-walker step): " + orc.describe(),
                "cpu_baseline": {"value": v, "unit": "walker-steps/s", "cores": orc.procs, "kind": "oracle",
                                 "sample": orc.describe()},
                "e2e": {"value": v, "unit": "walker-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t0}
        print(json_line(line))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        orc = OracleSample()
        r, slowest, steps = orc.run(0)
        orc.close()
        cpu = {"value": r, "unit": "walker-steps/s", "cores": orc.procs, "kind": "oracle",
               "sample": orc.describe() + f"; {time.perf_counter() - t0:.1f} s wall with process start-up"}
    res = run_gpu(args, rank, world)
    if rank == 0:
        peak = FP64_PEAK_GFLOPS
        fp64 = measure_fp64_peak(int(os.environ.get("LOCAL_RANK", 0)))
        measured = fp64.get("dfma_gflops")
        mixed = res["mixed"]
        line = {
            "metric": metric, "value": res["value"], "unit": "walker-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["step_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload,
            "electron_move_attempts_per_s": res["value"] * 6 * 16,
            "roofline": {"bound": "alu", "kernel": "k_propagate", "achieved": res["achieved"], "peak": peak,
                         "unit": "GFLOP/s (FP64 operations x 2, functions at their FP64 instruction count)",
                         "frac": res["achieved"] / peak, "traffic": PROPAGATE_TRAFFIC_BYTES,
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "peak_source": "nominal FP64 rate of the recipe table (the largest of the three FP64 "
                                        "peaks here; MEASURED_PEAKS has no FP64 entry)",
                         "kernel_ms": res["prop_ms"], "fp64_ops_per_walker_step": res["slots"],
                         "fp64_pipe_busy_ncu": PROPAGATE_FP64_PIPE_BUSY,
                         "fp64_warp_inst_per_walker_step_ncu": PROPAGATE_FP64_INST_PER_STEP,
                         "fp64_active_lanes_ncu": PROPAGATE_FP64_ACTIVE_LANES,
                         "peak_unit_count": FP64_UNIT_COUNT_GFLOPS,
                         "frac_vs_unit_count": res["achieved"] / FP64_UNIT_COUNT_GFLOPS,
                         "peak_measured_dfma": measured,
                         "frac_vs_measured_dfma": res["achieved"] / measured if measured else None,
                         "fp64_peak_run": fp64},
            "conventional": {"value": res["conv_rate"], "unit": "walker-steps/s", "tau": res["tau"],
                             "moves_mean_max": res["conv_moves"],
                             "lb_speedup": res["value"] / res["conv_rate"]},
            "load_imbalance": res["imbalance"],
            "cpu_baseline": cpu,
            "e2e": {"value": res["e2e"], "unit": "walker-steps/s", "h2d_bytes_per_step": res["h2d"],
                    "d2h_bytes_per_step": res["d2h"]},
            "mixed": dict(mixed, speedup_vs_fp64=mixed["value"] / res["value"]) if mixed else None,
            "fp64_51200": mixed["n_w_51200"]["fp64_value"] if mixed else None,
            "mixed_51200": mixed["n_w_51200"]["value"] if mixed else None,
            "mixed_speedup_51200": mixed["n_w_51200"]["speedup_vs_fp64"] if mixed else None,
            "mixed_bias_mHa": mixed["energy_bias_mHa"] if mixed else None,
            "mixed_bias_err_mHa": mixed["energy_bias_err_mHa"] if mixed else None,
            "tensor_core_51200": {k: {"value": v["value_51200"], "bias_mHa": v["energy_bias_mHa"],
                                      "bias_err_mHa": v["energy_bias_err_mHa"]}
                                  for k, v in mixed["tensor_core"].items()} if mixed else None,
            "a_scan": res["a_scan"],
            "h2_run": res["h2"],
            "batch": res["batch"],
            "adjoint": res["adjoint"],
            "large_systems": res["large"],
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
            "energy_unequilibrated": {"E": res["energy"][0], "err": res["energy"][1],
                                      "note": "estimator over the bench's ~30 water-methane intervals: not "
                                              "equilibrated (the synthetic Hamiltonian's ground state lies far "
                                              "below the random-MO trial function); the H2 sections give "
                                              "converged energies"},
        }
        print(json_line(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
