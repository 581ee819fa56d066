#!/usr/bin/env python
"""Benchmark of the nodal DG hot path: LSRK4-stage DOF-updates/s on GB300.

A step is one full low-storage RK4 step (five fused right-hand-side + stage
updates) of the workload, through libdg's C ABI.  The default workload is the
viscous configuration: compressible Navier-Stokes with BR1, mu = 1e-3,
Pr = 0.71, periodic box of 24^3 hexahedra x 6 = 82,944 tetrahedra, order N = 3
(20 nodes each), Taylor-Green vortex at Mach 0.1 with 1% seeded noise, FP64.
A DOF is one node of one element (per scalar field, as the paper counts them);
one stage updates K*Np DOFs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--config NAME]

One JSON line is printed by rank 0.  --impl reference times the FP64 CPU oracle
on the host cores instead (the reference arm).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The oracle's CPU timings run on one thread, its numpy BLAS calls included, so that the core
# count they report is the one they used (set before numpy is first imported).
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")


def host_cpu():
    """The host beside a CPU timing: architecture, logical CPUs, and the model where the kernel
    names one."""
    import platform
    info = {"machine": platform.machine(), "nproc": os.cpu_count()}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    info["model"] = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return info

METRIC = "RK4 stage DOF-updates/s on 1 GB300: mixed/learned vs plain FP64 at fixed error"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (2 FMA lanes x 152 SMs x 2.07 GHz x 2); the run measures it too
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture, keyed by the
# sha256 of the kernel sources they were taken on, the workload and the kernel; a changed kernel or
# another workload reports null traffic.
FP64_SOURCES = ("dg_kernels.cuh", "k_ns.cu", "k_euler.cu")
MIXED_SOURCES = ("dg_mixed.cuh", "dg_tc.cuh", "dg_umma.cuh", "dg_cvt.cuh", "dg_kernels.cuh", "k_mixed.cu", "k_tc.cu")
TRAFFIC = {
    # profiles/ns_N3_K82944_fp64.md and profiles/mixed_tc_ns_N3_K82944.md: DRAM read + write per
    # launch, mean over the five stages of one RK4 step
    ("276e74aec8aa44ec", "ns_viscous", "rhs"): 317.652700e6 + 105.683300e6,
    ("276e74aec8aa44ec", "ns_viscous", "viscous"): 126.923400e6 + 75.355550e6,
    ("276e74aec8aa44ec", "ns_viscous", "prims"): 66.387510e6 + 6.057626e6,
    ("9cd242f4cd10185f", "ns_viscous", "mixed_rhs"): 258.499700e6 + 95.220530e6,
    ("9cd242f4cd10185f", "ns_viscous", "mixed_viscous"): 90.070680e6 + 23.047480e6,
    ("9cd242f4cd10185f", "ns_viscous", "mixed_prims"): 66.372200e6 + 12.271460e6,
}


def kernel_source_hash(files=FP64_SOURCES):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2512_17101_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# The paper's own right-hand-side throughput figures (Sec. 5.3), with their hardware: context only
# (other hardware, a 2-D p = 1 tensor-product shock/boundary-layer case, no stated precision).
PAPER_CONTEXT = [
    {"figure": "RHS throughput", "value": 1.6e6, "unit": "DOFs/s", "hardware": "Apple M2 (CPU)",
     "case": "shock/boundary-layer Navier-Stokes, 2M p = 1 tensor-product elements (8M DOFs)"},
    {"figure": "RHS throughput", "value": 100.4e6, "unit": "DOFs/s", "hardware": "AMD MI300A (1 device)",
     "case": "same case"},
]

# ---- algorithmic work per launch ------------------------------------------------------------

def rhs_flops_per_element(Np, NF, V, viscous):
    """FP64 flops the fused right-hand side + stage update needs per element."""
    f = 2 * 3 * Np * Np * V          # -sum_a D_a F_a
    f += 2 * NF * Np * V             # LIFT g
    f += Np * V * 3 * 5              # contravariant fluxes
    f += Np * 30                     # pressure, velocity, Euler fluxes
    f += NF * (56 + 4 + 5 * V)       # both traces' p, c, u.n, n.F; lambda; LF flux and Fscale
    f += Np * V * 4                  # k <- a k + dt rhs, q <- q + b k
    if viscous:
        f += Np * 12 + NF * 48       # subtract viscous flux; central viscous normal flux
    return f


def viscous_flops_per_element(Np, NF):
    f = 2 * 3 * Np * Np * 5          # reference derivatives of (rho, rho u, T)
    f += Np * 5 * 3 * 5              # to physical gradients
    f += 2 * NF * Np * 5 + Np * 4 * 3 * 5 * 2  # lifted central jumps, per-face normals
    f += NF * 30 + Np * 15           # traces and T at own nodes
    f += Np * 60                     # velocity gradient, stress, heat flux
    return f


def rhs_bytes_per_element(Np, NF, V, viscous):
    b = Np * 8 * 4 * V + 26 * 8 + 4 * NF  # q, k in; q_out, k out; geometry; neighbour map
    b += Np * 8 * 3                        # the primitives pass's (1/rho, p, c)
    if viscous:
        b += Np * 8 * 9                    # viscous flux in
    return b


def viscous_bytes_per_element(Np, NF):
    return Np * 8 * (5 + 9 + 2) + 26 * 8 + 4 * NF  # q in, flux out, (1/rho, p) in; geometry; map


def prims_bytes_per_element(Np):
    return Np * 8 * (5 + 3)  # q in, (1/rho, p, c) out


# ---- clocks ------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", self.gpu], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- distributed plumbing ------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- oracle timing (the reference arm and the cpu_baseline leg) ------------------------------------

def oracle_stage_runner(cfg, n=None):
    """Returns (run_one_stage, dofs_per_stage, description) for the oracle on the config."""
    import numpy as np
    from oracle.euler import rhs_strong
    from oracle.geometry import connect, geometric_factors
    from oracle.lsrk import lsrk4_stage
    from oracle.ns import rhs_ns
    from oracle.refelem import build_reference
    from oracle.thermo import PerfectGas
    from workloads.configs import build_case
    case = build_case(cfg, n=n)
    ref = build_reference(cfg.N, case["ref_nodes"])
    geo = geometric_factors(case["vertices"])
    conn = connect(case["vertices"], case["period"], ref)
    gas = PerfectGas(cfg.gas.gamma, cfg.gas.R)
    if cfg.physics == "ns":
        f = lambda u: rhs_ns(ref, geo, conn, u, gas, cfg.gas.mu, cfg.gas.Pr)
    elif cfg.physics == "euler":
        f = lambda u: rhs_strong(ref, geo, conn, u, gas)
    else:
        raise ValueError(f"no oracle timing for {cfg.physics}")
    state = {"q": case["q"], "k": np.zeros_like(case["q"]), "s": 0}

    def run():
        state["q"], state["k"] = lsrk4_stage(state["q"], state["k"], state["s"], cfg.dt, f)
        state["s"] = (state["s"] + 1) % 5

    K = case["vertices"].shape[0]
    return run, K * ref.Np, f"one LSRK4 stage on {K} tets (box {case['n']}^3 x 6), N={cfg.N}"


def time_oracle(cfg, stages, n=None):
    run, dofs, desc = oracle_stage_runner(cfg, n)
    t0 = time.perf_counter()
    for _ in range(stages):
        run()
    dt = time.perf_counter() - t0
    return dofs * stages / dt, desc, dt


def _oracle_chunk_worker(cfg_name, n, lo, hi, local, out_faces, barrier, results):
    """One process of the all-core oracle timing: the oracle's LSRK4 stage on element range
    [lo, hi) of the workload (box side n), computed on a local mesh of the range plus its face
    neighbours two deep (faces leading out of the local set are outflow faces; two layers make the
    BR1 gradients of the first layer, and so the range's right-hand side, equal to the global ones).
    Waits on the barrier after its set-up and puts (lo, seconds of the stage, the range's RK
    register) on the results queue."""
    import numpy as np
    import oracle.boundary as bd
    from oracle.geometry import connect, geometric_factors
    from oracle.lsrk import lsrk4_stage
    from oracle.refelem import build_reference
    from oracle.thermo import PerfectGas
    from workloads.configs import build_case, get_config
    cfg = get_config(cfg_name)
    case = build_case(cfg, n=n)
    v = case["vertices"][local]
    ref = build_reference(cfg.N, case["ref_nodes"])
    period = np.asarray(case["period"], dtype=float)
    face_bc = np.zeros((len(local), 4), dtype=np.int32)
    face_bc[out_faces[:, 0], out_faces[:, 1]] = 4  # outflow
    geo = geometric_factors(v)
    conn = connect(v, period, ref, face_bc=face_bc)
    gas = PerfectGas(cfg.gas.gamma, cfg.gas.R)
    if cfg.physics == "ns":
        f = lambda u: bd.rhs_ns_bc(ref, geo, conn, u, gas, cfg.gas.mu, cfg.gas.Pr)
    else:
        f = lambda u: bd.rhs_euler_bc(ref, geo, conn, u, gas)
    q = np.ascontiguousarray(case["q"][:, local])
    k = np.zeros_like(q)
    barrier.wait(timeout=1800)
    t0 = time.perf_counter()
    _, k1 = lsrk4_stage(q, k, 0, cfg.dt, f)
    results.put((lo, time.perf_counter() - t0, np.ascontiguousarray(k1[:, : hi - lo])))


def oracle_all_cores(cfg, cores, n=None):
    """The oracle's LSRK4 stage (stage 0) on the workload, the elements split into `cores` contiguous
    ranges, one spawned process per range (element-parallel, the analogue of an OpenMP loop over
    elements for a numpy program).  Returns (DOF-updates/s, seconds of the slowest process,
    description, the RK register [V][K][Np] assembled from the ranges)."""
    import multiprocessing as mp
    import numpy as np
    from paper_2512_17101_gb300 import dg
    from workloads.configs import build_case
    case = build_case(cfg, n=n)
    K = case["vertices"].shape[0]
    glob = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"], host_only=True)
    E, _ = glob.face_pairs()
    ctx = mp.get_context("spawn")
    bar, results = ctx.Barrier(cores), ctx.Queue()
    procs = []
    for r in range(cores):
        lo, hi = K * r // cores, K * (r + 1) // cores
        owned = np.arange(lo, hi)
        ring1 = np.setdiff1d(np.unique(E[owned][E[owned] >= 0]), owned)
        ring2 = np.setdiff1d(np.unique(E[ring1][E[ring1] >= 0]), np.concatenate([owned, ring1]))
        local = np.concatenate([owned, ring1, ring2])
        pos = np.full(K, -1)
        pos[local] = np.arange(len(local))
        nb = E[local]
        out = np.argwhere((nb >= 0) & (pos[np.maximum(nb, 0)] < 0))
        p = ctx.Process(target=_oracle_chunk_worker, args=(cfg.name, n, lo, hi, local, out, bar, results))
        p.start()
        procs.append(p)
    got = [results.get(timeout=3600) for _ in range(cores)]
    for p in procs:
        p.join()
    secs = max(t for _, t, _ in got)
    k = np.concatenate([kk for _, _, kk in sorted(got, key=lambda x: x[0])], axis=1)
    value = K * glob.Np / secs
    desc = (f"one LSRK4 stage on {K} tets (box {case['n']}^3 x 6), N={cfg.N}, in {cores} element ranges, one "
            f"process per core, each with a two-element-deep halo (its range's stage equals the "
            f"single-process one); the slowest process's time, set-up excluded")
    return value, secs, desc, k


def reference_arm(args, cfg, world, rank):
    if rank != 0:
        return
    sub_n = max(2, cfg.n // 2)
    run, dofs, desc = oracle_stage_runner(cfg, n=sub_n)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    el = time.perf_counter() - t0
    value = dofs * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(cfg), timed_on=f"{desc}: the workload's order, physics and state recipe on "
                                                          f"a box of half its side (DOF-updates/s is a per-DOF "
                                                          f"rate; the full box takes ~8x longer per stage)"),
        "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": 1, "host": host_cpu(), "kind": "oracle",
                         "sample": f"each step: {desc} (half-size box of the workload); numpy, single thread"},
        "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(cfg):
    return {"workload": f"{cfg.name}: {cfg.description}", "K": cfg.K, "N": cfg.N, "Np": cfg.Np,
            "V": 5, "physics": cfg.physics, "dofs_per_stage": cfg.dofs, "stages_per_step": 5,
            "dt": cfg.dt, "precision": cfg.precision,
            "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


# ---- GPU arm -------------------------------------------------------------------------------------

def mixed_prims_bytes_per_element(Np, viscous):
    """q in (FP64); the 32-byte node record (float state, pressure and density as hi/lo pairs) and,
    for Navier-Stokes, the temperature pair out."""
    return Np * (40 + 32 + (8 if viscous else 0))


def mixed_rhs_bytes_per_element(Np, NF, viscous):
    """node records in; q in, k in/out, q_out (FP64); fp32 geometry; neighbour map."""
    b = Np * (32 + 4 * 40) + 26 * 4 + 4 * NF
    if viscous:
        b += Np * 4 * 9                      # fp32 viscous-flux record in
    return b


def mixed_viscous_bytes_per_element(Np, NF):
    """node records and temperature pairs in; fp32 viscous-flux record out; fp32 geometry; neighbour map."""
    return Np * (32 + 8 + 36) + 26 * 4 + 4 * NF


def mixed_tensor_flops_per_element(Np, NF, viscous):
    """Tensor-core flops of the split-BF16 products (6 products per contraction, real rows and columns)."""
    f = 6 * 2 * 5 * Np * (3 * Np + NF)                        # [-D_r -D_s -D_t | LIFT] contraction
    if viscous:
        f += 6 * 2 * 5 * 3 * Np * (Np + NF)                   # BR1: [D_a | Lhat_a], a = r, s, t
    return f


def gpu_arm(args, cfg, world, rank, local):
    import numpy as np
    import torch
    from paper_2512_17101_gb300 import capi, dg
    from workloads.configs import build_case

    if not os.path.exists(capi.LIB_PATH):
        raise SystemExit("libdg.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = build_case(cfg)
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"])
    g = cfg.gas
    gas = dg.Gas(model="perfect", gamma=g.gamma, R=g.R, mu=g.mu, Pr=g.Pr)
    q0 = torch.tensor(case["q"], device=dev)
    work = (torch.empty_like(q0), torch.zeros_like(q0))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    forms = {"fp64": dg._opts(precision=capi.DG_PREC_FP64), "mixed": dg._opts(precision=capi.DG_PREC_MIXED)}

    def step(qbuf, form):
        dg.lsrk4_step(mesh, gas, qbuf, cfg.dt, steps=1, work=work, opts=forms[form])

    def timed_run(form, with_clocks):
        q = q0.clone()
        for _ in range(args.warmup):
            step(q, form)
        q.copy_(q0)
        torch.cuda.synchronize()
        mesh.kernel_times(reset=True)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(local) if with_clocks else None
        mesh.set_timing(True)
        barrier(world)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev0[i].record(stream)
            step(q, form)
            ev1[i].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clock_info = clocks.stop() if clocks else None
        mesh.set_timing(False)
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)), world)
        ktimes = mesh.kernel_times(reset=True)
        if mesh.status() != 0:
            raise SystemExit(f"device status flags set during the {form} run (non-physical state)")
        return dict(ms=total_ms / args.steps, ktimes=ktimes, clocks=clock_info, q=q)

    head = args.precision
    other = "mixed" if head == "fp64" else "fp64"
    runs = {head: timed_run(head, True), other: timed_run(other, False)}
    q_one = q0.clone()
    step(q_one, head)
    runs[head]["q_one"] = q_one  # one step from the initial state: what every end-to-end step returns
    dofs_step = cfg.dofs * 5
    Np, NF = cfg.Np, 4 * ((cfg.N + 1) * (cfg.N + 2) // 2)
    viscous = g.mu > 0

    def kernel_table(ktimes):
        per = {name: {"avg_ms": ms / n, "launches": n} for name, (ms, n) in ktimes.items() if n}
        tot = sum(v["avg_ms"] * v["launches"] for v in per.values())
        for v in per.values():
            v["share"] = v["avg_ms"] * v["launches"] / tot
        return per

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp64_measured = dg.dg_fp64_fma_rate()
    src = kernel_source_hash(FP64_SOURCES)
    src_mixed = kernel_source_hash(MIXED_SOURCES)

    def roofline(form, per):
        dom = max(per, key=lambda k: per[k]["avg_ms"] * per[k]["launches"])
        avg_s = per[dom]["avg_ms"] * 1e-3
        if form == "fp64":
            for name, fn in (("rhs", lambda: rhs_bytes_per_element(Np, NF, 5, viscous)),
                             ("viscous", lambda: viscous_bytes_per_element(Np, NF)),
                             ("prims", lambda: prims_bytes_per_element(Np))):
                if name in per:
                    per[name]["algorithmic_bytes"] = fn() * cfg.K
                    per[name]["traffic"] = TRAFFIC.get((src, cfg.name, name))
            if dom == "rhs":
                flops = rhs_flops_per_element(Np, NF, 5, viscous) * cfg.K
                nbytes = rhs_bytes_per_element(Np, NF, 5, viscous) * cfg.K
            else:
                flops = viscous_flops_per_element(Np, NF) * cfg.K
                nbytes = viscous_bytes_per_element(Np, NF) * cfg.K
            ach = flops / avg_s / 1e12
            return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS, "traffic": TRAFFIC.get((src, cfg.name, dom)), "kernel": dom,
                    "flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                    "fp64_fma_measured_tflops": fp64_measured,
                    "frac_of_measured_fp64": ach / fp64_measured if fp64_measured else None,
                    "hbm_achieved_gbs": nbytes / avg_s / 1e9, "hbm_peak_gbs": hbm_peak,
                    "hbm_frac": nbytes / avg_s / 1e9 / hbm_peak, "kernels": per,
                    "peak_note": "FP64 nominal 1.25 TFLOP/s (2 FMA lanes x 152 SMs x 2.07 GHz); beside it the "
                                 "FP64 FMA rate measured in this run by the library's probe kernel "
                                 "(dg_fp64_fma_rate); HBM: measured copy"}
        per_el = {"rhs": mixed_rhs_bytes_per_element(Np, NF, viscous),
                  "viscous": mixed_viscous_bytes_per_element(Np, NF),
                  "prims": mixed_prims_bytes_per_element(Np, viscous)}
        for name, v in per.items():
            if name in per_el:
                v["algorithmic_bytes"] = per_el[name] * cfg.K
                v["hbm_frac"] = per_el[name] * cfg.K / (v["avg_ms"] * 1e-3) / 1e9 / hbm_peak
        nbytes = per_el[dom] * cfg.K
        ach = nbytes / avg_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": TRAFFIC.get((src_mixed, cfg.name, "mixed_" + dom)), "kernel": dom,
                "algorithmic_bytes_per_launch": nbytes,
                "tensor_flops_per_step": mixed_tensor_flops_per_element(Np, NF, viscous) * cfg.K * 5,
                "kernels": per, "peak_note": "HBM: measured copy (MEASURED_PEAKS.json)"}

    # mixed form's error against the fp64 form after the same steps from the same state
    qa, qb = runs["fp64"]["q"], runs["mixed"]["q"]
    comp = [float(((qb[v] - qa[v]).abs().max() / qa[v].abs().max()).item()) for v in range(5)]
    mom = float((qb[1:4] - qa[1:4]).abs().max().item() / qa[1:4].abs().max().item())
    field = max(comp[0], mom, comp[4])
    mom_max = float(qa[1:4].abs().max().item())
    significant = [v for v in range(5) if v not in (1, 2, 3) or float(qa[v].abs().max().item()) >= 0.01 * mom_max]
    comp_sig = max(comp[v] for v in significant)
    abs_err = [float((qb[v] - qa[v]).abs().max().item()) for v in range(5)]

    per_head = kernel_table(runs[head]["ktimes"])
    per_other = kernel_table(runs[other]["ktimes"])
    ms_per_step = runs[head]["ms"]
    value = world * dofs_step / (ms_per_step * 1e-3)
    other_line = {"precision": other, "value": world * dofs_step / (runs[other]["ms"] * 1e-3),
                  "unit": "DOF-updates/s", "ms_per_step": runs[other]["ms"],
                  "roofline": roofline(other, per_other)}
    mixed_err = {"vs": "fp64 form on the same state (the fp64 form matches the oracle to 1e-11, tests/test_gpu_parity.py)",
                 "steps": args.steps, "per_field_max": field, "per_component": comp,
                 "per_component_abs": abs_err, "per_component_max_over_significant": comp_sig,
                 "components_significant": significant,
                 "definition": "per_field_max (the bar, <= 1e-6): max over the fields rho, momentum as one vector, "
                               "rho E of max|a - b| / max|b|; per_component: max|a_v - b_v| / max|b_v| for each "
                               "component; significant components have a maximum >= 1 % of their field's (rho w "
                               "stays near zero from the w = 0 Taylor-Green start, so its own-relative error is set "
                               "by the rounding of the other components)"}

    # end to end through the public API, as a loop over independent states would run it: every step
    # copies its input in from pinned host memory, takes one RK4 step and copies its result back.
    # The device state is double-buffered, so the next step's input copy and the previous step's
    # result copy run on two copy streams while a step computes; the timed region runs from before
    # the first input copy to the end of the last result copy.
    qb = [q0.clone(), q0.clone()]
    host_in = torch.empty(q0.shape, dtype=torch.float64, pin_memory=True)
    host_in.copy_(q0.cpu())
    host_out = [torch.empty_like(host_in, pin_memory=True) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    in_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    step_done = [torch.cuda.Event() for _ in range(2)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t0.record(stream)
    s_in.wait_event(t0)
    for i in range(args.steps):
        b = i % 2
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(out_done[b])  # the buffer's previous result is on the host
            qb[b].copy_(host_in, non_blocking=True)
            in_done[b].record(s_in)
        flush.fill_(float(i))
        stream.wait_event(in_done[b])
        step(qb[b], head)
        step_done[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(step_done[b])
            host_out[b].copy_(qb[b], non_blocking=True)
            out_done[b].record(s_out)
    stream.wait_event(out_done[(args.steps - 1) % 2])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(t0.elapsed_time(t1), world) / args.steps
    ref1 = runs[head]["q_one"].cpu()
    if (host_out[(args.steps - 1) % 2] - ref1).abs().max() > 1e-12 * ref1.abs().max():
        raise SystemExit("the end-to-end step's result differs from a step of the same state on the device")
    state_bytes = q0.numel() * 8
    e2e = {"value": world * dofs_step / (e2e_ms * 1e-3), "unit": "DOF-updates/s",
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes, "ms_per_step": e2e_ms,
           "copies": "double-buffered device state; the next input's and the previous result's copies "
                     "overlap a step on two copy streams"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, desc, secs = time_oracle(cfg, 1)
        cpu = {"value": val, "unit": "DOF-updates/s", "cores": 1, "host": host_cpu(), "kind": "oracle",
               "sample": f"{desc}: the full workload's mesh; numpy, single thread; {secs:.1f} s"}
        ncores = os.cpu_count() or 1
        if ncores > 1:
            vall, secs_all, desc_all, _ = oracle_all_cores(cfg, ncores)
            cpu["all_cores"] = {"value": vall, "unit": "DOF-updates/s", "cores": ncores, "kind": "oracle",
                                "sample": f"{desc_all}; {secs_all:.2f} s"}

    learned = None
    if rank == 0 and not args.no_learned:
        learned = learned_form(args, local)
    batched = None
    if rank == 0 and not args.no_batched:
        batched = batched_form(args, local)
    hexf = hexadv = hexshock = None
    if rank == 0 and not args.no_hex:
        hexf = hex_form(args, local)
        hexadv = hex_advection_form(args, local)
        hexshock = hex_shock_form(args, local)
    bnd = avf = mixns = None
    if rank == 0 and not args.no_boundary:
        periodic = value if (head == "fp64" and cfg.name == "ns_viscous") else None
        bnd = boundary_form(args, local, periodic)
        avf = av_form(args, local)
        mixns = mixture_ns_form(args, local)
    oif = None
    if rank == 0 and not args.no_overint:
        oif = overint_form(args, local)
    partf = None
    if rank == 0 and not args.no_partitioned:
        partf = partitioned_form(args, local, runs["fp64"]["ms"] if cfg.name == "ns_viscous" else None)
    launches = sum(v["launches"] for v in per_head.values())
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f64 state; bf16x3 tensor / fp32 flux",
            "data": "synthetic", "config": dict(workload_config(cfg), precision=head),
            "roofline": roofline(head, per_head), "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": runs[head]["clocks"], "other_form": other_line, "mixed_error": mixed_err,
            "learned_form": learned, "batched_form": batched, "hex_form": hexf,
            "paper_context": PAPER_CONTEXT,
            "hex_advection_form": hexadv, "hex_shock_form": hexshock, "boundary_form": bnd, "av_form": avf, "mixture_ns_form": mixns,
            "partitioned_form": partf, "overint_form": oif, "kernel_src": {"fp64": src, "mixed": src_mixed},
            "impl": "gpu",
        }
        print(json.dumps(line), flush=True)


# nonzeros of the three modal derivative matrices V_o^-1 D_a V_o of the orthonormal tetrahedral
# basis, by order (their zero pattern is structural: a mode's derivative has lower degree)
MODAL_DERIVATIVE_NNZ = {1: 6, 2: 46, 3: 202, 4: 647}


def overint_flops_per_element(N, Q, viscous=False):
    """FP64 flops of one element in the sum-factorised over-integrated right-hand side (Q points
    per collapsed direction, Q^3 in all; an FMA counts two): the modes (V_o^-1 on 5 fields), the
    three 1-D sums to the points, per point the state's last sum and the Euler flux (about 30), the
    three weighted 1-D sums back for the 15 flux components (the first folded by the symmetry of
    the Gauss-Legendre points), the moments' contravariant transform
    (15 per mode and field), the sparse modal derivative matrices, V_o and LIFT; about 100 per face
    node for the Lax-Friedrichs flux.  Viscous: the nodal contravariant viscous flux (75 per node),
    the modes of its four rows (V_o^-1 for each direction), and about 40 more per face node for the
    central viscous flux."""
    Np, Nfp = (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2
    NF, Nt2, q2, q3 = 4 * Nfp, Nfp, Q * Q, Q ** 3
    f = 2 * 5 * Np * Np + 2 * 5 * Q * Np + 2 * 5 * q2 * Nt2
    f += q3 * (2 * 5 * (N + 1) + 30)
    h = Q // 2  # the backward a-sum folds the symmetric Gauss-Legendre points: per line 2h sums, then
    # h FMAs per mode p and the middle point for even p
    f += 15 * q2 * (2 * h + 2 * (N + 1) * h + 2 * ((N + 2) // 2) * (Q % 2))
    f += 2 * 15 * Nt2 * q2 + 5 * Np * (2 * 3 * Q + 15)
    f += 2 * 5 * MODAL_DERIVATIVE_NNZ[N] + 2 * 5 * Np * (Np + NF) + 100 * NF
    if viscous:
        f += 75 * Np + 2 * 4 * 3 * Np * Np + 40 * NF
    return f


def overint_form(args, local):
    """Over-integration (weak form, Stroud rule with ceil(3N/2) points per collapsed direction) on the
    periodic vortex with the main workload's mesh and order (24^3 x 6 tets, N = 3), Euler and
    Navier-Stokes (mu = 1e-3, Pr = 0.71): FP64 RK4 steps with CUDA events, against the collocated
    strong form on the same mesh, and the over-integrated kernel's FP64 rate from its flop count."""
    import torch
    from paper_2512_17101_gb300 import dg
    from workloads import box_mesh, equispaced_tet_nodes, isentropic_vortex, physical_nodes, uniform_perturbation

    n, N = 24, 3
    dev = torch.device("cuda", local)
    v, per = box_mesh(n, 1.0)
    nodes = equispaced_tet_nodes(N)
    mesh = dg.Mesh(v, per, N, nodes)
    q0 = torch.tensor(uniform_perturbation(isentropic_vortex(physical_nodes(v, nodes), 0.0), 1e-3, seed=0),
                      device=dev)
    K, Np = v.shape[0], nodes.shape[0]
    dt = 1e-4
    work = (torch.empty_like(q0), torch.zeros_like(q0))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    steps = max(1, min(args.steps, 10))
    out = {}
    for label, oq, mu in (("collocated", 0, 0.0), ("overint", -1, 0.0), ("ns_collocated", 0, 1e-3),
                          ("ns_overint", -1, 1e-3)):
        gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=mu, Pr=0.71)
        mesh.set_overint(oq)
        q = q0.clone()
        for _ in range(max(3, args.warmup)):
            dg.lsrk4_step(mesh, gas, q, dt, steps=1, work=work)
        q.copy_(q0)
        total = 0.0
        mesh.kernel_times(reset=True)
        mesh.set_timing(True)
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dg.lsrk4_step(mesh, gas, q, dt, steps=1, work=work)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
        mesh.set_timing(False)
        kt = mesh.kernel_times(reset=True)
        if mesh.status() != 0:
            raise SystemExit("status flags set in the over-integration run")
        ms = total / steps
        out[label] = {"ms_per_step": ms, "value": K * Np * 5 / (ms * 1e-3),
                      "rhs_avg_ms": kt["rhs"][0] / kt["rhs"][1] if kt["rhs"][1] else None}
    Q = (3 * N + 1) // 2

    def roof(viscous):
        flops = overint_flops_per_element(N, Q, viscous) * K
        ach = flops / (out["ns_overint" if viscous else "overint"]["rhs_avg_ms"] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": "rhs_oi_kernel", "flops_per_launch": flops, "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "peak_kind": "nominal FP64"}

    return {
        "workload": f"periodic isentropic vortex + U(+-1e-3), {n}^3 x 6 = {K} tets, N = {N}, FP64; "
                    "Euler and Navier-Stokes (mu = 1e-3, Pr = 0.71)",
        "points_per_direction": Q, "points_per_element": Q ** 3, "unit": "DOF-updates/s", **out,
        "slowdown": out["overint"]["ms_per_step"] / out["collocated"]["ms_per_step"],
        "ns_slowdown": out["ns_overint"]["ms_per_step"] / out["ns_collocated"]["ms_per_step"],
        "roofline": roof(False), "ns_roofline": roof(True),
    }


def learned_form(args, local):
    """The learned form's workload (7-species Euler mixture, 32^3 x 6 tets, N = 2): RK4 steps with the
    Newton temperature solve seeded by a constant, by the previous stage's T, and by the trained MLP."""
    import numpy as np
    import torch
    from paper_2512_17101_gb300 import capi, dg
    from workloads.configs import build_case, get_config
    from workloads.mlp import glorot_params, temperature_samples

    cfg = get_config("mixture_learned")
    dev = torch.device("cuda", local)
    case = build_case(cfg)
    mix = case["mixture"]
    gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50)
    K, Np = case["vertices"].shape[0], case["ref_nodes"].shape[0]
    n = K * Np
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"])
    # conserved state from (Y, T, u, p0): density from the mixture gas constant, energy from the library's EOS
    Y = np.ascontiguousarray(case["Y"].reshape(7, n))
    T = np.ascontiguousarray(case["T"].reshape(n))
    vel = np.ascontiguousarray(case["vel"].reshape(3, n))
    Rmix = (Y * (mix.R_universal / mix.W)[:, None]).sum(axis=0)
    rho = case["p0"] / (Rmix * T)
    Yd, Td = torch.tensor(Y, device=dev), torch.tensor(T, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev)
    dg.dg_mixture_energy(gas, Td, Yd, e)
    rho_d, vel_d = torch.tensor(rho, device=dev), torch.tensor(vel, device=dev)
    q0 = torch.empty((12, n), dtype=torch.float64, device=dev)
    q0[0] = rho_d
    q0[1:4] = rho_d * vel_d
    q0[4] = rho_d * (e + 0.5 * (vel_d * vel_d).sum(dim=0))
    q0[5:] = rho_d * Yd
    q0 = q0.reshape(12, K, Np).contiguous()

    # training data: uniform T, Dirichlet Y -> e (library EOS) -> Newton labels from a constant seed
    t0 = time.perf_counter()
    Ts, Ys = temperature_samples(1_000_000, 7, seed=7)
    Tsd, Ysd = torch.tensor(Ts, device=dev), torch.tensor(Ys, device=dev)
    es = torch.empty_like(Tsd)
    dg.dg_mixture_energy(gas, Tsd, Ysd, es)
    qs = torch.zeros((12, Ts.size), dtype=torch.float64, device=dev)
    qs[0], qs[4], qs[5:] = 1.0, es, Ysd
    Tl = torch.full_like(Tsd, 1650.0)
    dg.dg_temperature(gas, qs, Tl)
    torch.cuda.synchronize()
    hist = dg.dg_mlp_train(gas, es, Ysd, Tl, glorot_params(0), epochs=30, batch=1024, lr=3e-3, lr_decay=0.9)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    seed_modes = {"constant_1650K": (capi.DG_TSEED_CONST, 1650.0), "previous_stage_T": (capi.DG_TSEED_INPUT, 0.0),
                  "mlp": (capi.DG_TSEED_MLP, 0.0)}
    precisions = {"fp64": capi.DG_PREC_FP64, "mixed": capi.DG_PREC_MIXED}
    out = {"fp64": {}, "mixed": {}}
    steps = max(2, min(args.steps, 5))
    for pname, prec in precisions.items():
        for name, (mode, tc) in seed_modes.items():
            opts = dg._opts(precision=prec, t_seed=mode, t_const=tc)
            q = q0.clone()
            Tio = torch.full((K, Np), 1650.0, dtype=torch.float64, device=dev)
            work = (torch.empty_like(q), torch.zeros_like(q))
            for _ in range(2):
                dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, T_io=Tio, opts=opts, work=work)
            q.copy_(q0)
            Tio.fill_(1650.0)
            torch.cuda.synchronize()
            mesh.kernel_times(reset=True)
            mesh.set_timing(True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=steps, T_io=Tio, opts=opts, work=work)
            b.record()
            torch.cuda.synchronize()
            mesh.set_timing(False)
            kt = mesh.kernel_times(reset=True)
            ms = a.elapsed_time(b) / steps
            # Newton iterations of one solve on the final state from this seed
            it = torch.zeros(n, dtype=torch.int32, device=dev)
            Tt = Tio.reshape(n).clone() if name == "previous_stage_T" else torch.empty(n, dtype=torch.float64, device=dev)
            dg.dg_temperature(gas, q.reshape(12, n), Tt, it, opts=dg._opts(t_seed=mode, t_const=tc))
            # the state after the workload's own step count, for the error bar
            q1 = q0.clone()
            T1 = torch.full((K, Np), 1650.0, dtype=torch.float64, device=dev)
            dg.lsrk4_step(mesh, gas, q1, cfg.dt, steps=cfg.steps, T_io=T1, opts=opts, work=work)
            r = {"ms_per_step": ms, "value": cfg.dofs * 5 / (ms * 1e-3), "unit": "DOF-updates/s",
                 "newton_iterations_mean": float(it.double().mean().item()), "q": q, "q1": q1}
            for kname in ("temperature", "prims", "rhs"):
                if kt[kname][1]:
                    r[kname + "_ms_per_stage"] = kt[kname][0] / kt[kname][1]
            out[pname][name] = r
            if gas.status() != 0 or mesh.status() != 0:
                raise SystemExit(f"status flags set in the learned-form run ({pname}, {name})")
    ref_q, ref_q1 = out["fp64"]["constant_1650K"]["q"], out["fp64"]["constant_1650K"]["q1"]

    def field_err(a_, b_):
        groups = [[0], [1, 2, 3], [4]] + [[v] for v in range(5, 12)]
        return max(float((a_[g] - b_[g]).abs().max().item() / b_[g].abs().max().item()) for g in groups)

    def per_variable(a_, b_):
        return [float((a_[v] - b_[v]).abs().max().item() / b_[v].abs().max().item()) for v in range(12)]

    for pname in out:
        for name in out[pname]:
            out[pname][name][f"state_err_vs_fp64_after_{cfg.steps}_step"] = field_err(out[pname][name]["q1"], ref_q1)
            out[pname][name][f"state_err_vs_fp64_after_{steps}_steps"] = field_err(out[pname][name]["q"], ref_q)
            out[pname][name][f"state_err_per_variable_after_{steps}_steps"] = per_variable(out[pname][name]["q"], ref_q)
    for pname in out:
        for name in out[pname]:
            out[pname][name].pop("q")
            out[pname][name].pop("q1")
    plain, combined = out["fp64"]["constant_1650K"], out["mixed"]["mlp"]
    return {"workload": f"{cfg.name}: {cfg.description}", "K": K, "N": cfg.N, "V": 12, "steps": steps,
            "training": {"samples": int(Ts.size), "epochs": 30, "seconds_incl_sampling": train_s,
                         "loss_first_last": [float(hist[0]), float(hist[-1])]},
            "mixed_plus_learned": {"value": combined["value"], "unit": "DOF-updates/s",
                                   "vs_plain_fp64_constant_seed": combined["value"] / plain["value"],
                                   "state_err_per_field": combined[f"state_err_vs_fp64_after_{cfg.steps}_step"],
                                   "state_err_per_field_after_timed_steps": combined[f"state_err_vs_fp64_after_{steps}_steps"],
                                   "error_measure": f"max over fields (rho, momentum vector, rho E, each rho Y_k) of "
                                                    f"max|q - q_fp64| / max|q_fp64| after the workload's {cfg.steps} RK4 "
                                                    f"step(s) from the same state; the per-node random mass fractions "
                                                    f"make the state move ~7 % per step, so the error grows ~linearly "
                                                    f"with the steps taken"},
            "seeds": out["fp64"], "mixed_precision_seeds": out["mixed"]}


def hex_flops_per_element(M):
    """FP64 flops of the sum-factorised hexahedral right-hand side + stage update per element (M = N+1)."""
    per_node = 8 + 21 + 2 * 3 * 5 * M + 4 * 5   # pressure, fluxes, 3 line derivatives x 5 vars (the
    #                                             -(2/h_d) dt factor folded into D), RK update
    per_face_node = 60                              # neighbour p, c, u.n, n.F of both traces, lambda, LF
    return M ** 3 * per_node + 6 * M * M * per_face_node


def hex_bytes_per_element(M):
    """q in, k in/out, q_out (FP64, 5 variables); neighbour traces assumed L2-resident."""
    return M ** 3 * 5 * 8 * 4


def hex_form(args, local):
    """The tensor-product hexahedron workload (Euler, isentropic vortex, 32^3 hexahedra, N = 4):
    FP64 RK4 steps with CUDA events, its FP64 roofline, and the oracle's stage on a 16^3 box."""
    import torch
    from paper_2512_17101_gb300 import dg
    from workloads.configs import build_hex_case, get_config

    cfg = get_config("hex_vortex")
    dev = torch.device("cuda", local)
    case = build_hex_case(cfg)
    mesh = dg.HexMesh(case["box"]["n"], case["box"]["L"], cfg.N, case["nodes1d"])
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0)
    q0 = torch.tensor(case["q"], device=dev)
    q = q0.clone()
    work = (torch.empty_like(q), torch.zeros_like(q))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        dg.hex_lsrk4_step(mesh, gas, q, cfg.dt, steps=1, work=work)
    q.copy_(q0)
    steps = max(1, args.steps)
    total = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.hex_lsrk4_step(mesh, gas, q, cfg.dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    if mesh.status() != 0:
        raise SystemExit("status flags set in the hexahedral run")
    ms = total / steps
    # the same steps with viscosity (Navier-Stokes, BR1, mu = 1e-3, Pr = 0.71)
    ns = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=1e-3, Pr=0.71)
    qn = q0.clone()
    for _ in range(max(3, args.warmup)):
        dg.hex_lsrk4_step(mesh, ns, qn, cfg.dt, steps=1, work=work)
    qn.copy_(q0)
    total_ns = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.hex_lsrk4_step(mesh, ns, qn, cfg.dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total_ns += a.elapsed_time(b)
    if mesh.status() != 0:
        raise SystemExit("status flags set in the hexahedral Navier-Stokes run")
    ms_ns = total_ns / steps
    # the Euler steps with over-integration (ceil(3 (N+1) / 2) Gauss points per axis)
    mesh.set_overintegration(True)
    qo = q0.clone()
    for _ in range(max(3, args.warmup)):
        dg.hex_lsrk4_step(mesh, gas, qo, cfg.dt, steps=1, work=work)
    qo.copy_(q0)
    total_oi = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.hex_lsrk4_step(mesh, gas, qo, cfg.dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total_oi += a.elapsed_time(b)
    if mesh.status() != 0:
        raise SystemExit("status flags set in the over-integrated hexahedral run")
    ms_oi = total_oi / steps
    # and the Navier-Stokes steps with over-integration
    qon = q0.clone()
    for _ in range(max(3, args.warmup)):
        dg.hex_lsrk4_step(mesh, ns, qon, cfg.dt, steps=1, work=work)
    qon.copy_(q0)
    total_oin = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.hex_lsrk4_step(mesh, ns, qon, cfg.dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total_oin += a.elapsed_time(b)
    mesh.set_overintegration(False)
    if mesh.status() != 0:
        raise SystemExit("status flags set in the over-integrated hexahedral Navier-Stokes run")
    ms_oin = total_oin / steps
    M = cfg.N + 1
    stage_s = ms * 1e-3 / 5
    flops, nbytes = hex_flops_per_element(M) * cfg.K, hex_bytes_per_element(M) * cfg.K
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    cpu = None
    if not args.no_cpu_baseline:  # the oracle's stage on a 16^3 box (one core), for context
        import oracle.hex as hx
        from oracle.thermo import PerfectGas
        small = build_hex_case(cfg, n=16)
        ref = hx.hex_reference(small["nodes1d"])
        t0 = time.perf_counter()
        hx.hex_rhs_strong(ref, small["box"], small["q"], PerfectGas(1.4, 1.0))
        cpu_s = time.perf_counter() - t0
        cpu = {"value": 16 ** 3 * M ** 3 / cpu_s, "unit": "DOF-updates/s", "cores": 1, "host": host_cpu(),
               "sample": f"one right-hand side of the oracle on 16^3 hexahedra, N = {cfg.N} "
                         f"(numpy, single thread), {cpu_s:.2f} s"}
    return {"workload": f"{cfg.name}: {cfg.description}", "K": cfg.K, "N": cfg.N, "Np": M ** 3, "dtype": "f64",
            "steps": steps, "ms_per_step": ms, "value": cfg.dofs * 5 / (ms * 1e-3), "unit": "DOF-updates/s",
            "roofline": {"bound": "alu", "achieved": flops / stage_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / stage_s / 1e12 / FP64_PEAK_TFLOPS,
                         "flops_per_stage": flops, "algorithmic_bytes_per_stage": nbytes,
                         "hbm_achieved_gbs": nbytes / stage_s / 1e9, "hbm_frac": nbytes / stage_s / 1e9 / hbm},
            "cpu_oracle_stage": cpu,
            "navier_stokes": {"mu": 1e-3, "Pr": 0.71, "ms_per_step": ms_ns,
                              "value": cfg.dofs * 5 / (ms_ns * 1e-3), "unit": "DOF-updates/s"},
            "overintegrated": {"gauss_points_per_axis": (3 * M + 1) // 2, "ms_per_step": ms_oi,
                               "value": cfg.dofs * 5 / (ms_oi * 1e-3), "unit": "DOF-updates/s",
                               "navier_stokes_ms_per_step": ms_oin},
            "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


def boundary_form(args, local, periodic_fp64=None):
    """The wall-bounded workload (Navier-Stokes channel, no-slip adiabatic walls at y = 0, 1,
    24^3 x 6 tets, N = 3): FP64 RK4 steps with CUDA events, the kernel split, against the
    periodic workload of the same size and order (the main line's FP64 value)."""
    import torch
    from paper_2512_17101_gb300 import dg
    from workloads.configs import build_case, get_config

    cfg = get_config("ns_channel")
    dev = torch.device("cuda", local)
    case = build_case(cfg)
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"], face_bc=case["face_bc"])
    g = cfg.gas
    gas = dg.Gas(model="perfect", gamma=g.gamma, R=g.R, mu=g.mu, Pr=g.Pr)
    q0 = torch.tensor(case["q"], device=dev)
    q = q0.clone()
    work = (torch.empty_like(q), torch.zeros_like(q))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, work=work)
    q.copy_(q0)
    steps = max(1, args.steps)
    total = 0.0
    mesh.kernel_times(reset=True)
    mesh.set_timing(True)
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    mesh.set_timing(False)
    kt = {name: {"avg_ms": ms / n, "launches": n} for name, (ms, n) in mesh.kernel_times(reset=True).items() if n}
    if mesh.status() != 0:
        raise SystemExit("status flags set in the wall-bounded run")
    ms = total / steps
    value = cfg.dofs * 5 / (ms * 1e-3)
    # the same steps in the mixed-precision form
    from paper_2512_17101_gb300 import capi
    mixed = dg._opts(precision=capi.DG_PREC_MIXED)
    qm = q0.clone()
    for _ in range(max(3, args.warmup)):
        dg.lsrk4_step(mesh, gas, qm, cfg.dt, steps=1, work=work, opts=mixed)
    qm.copy_(q0)
    total_m = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.lsrk4_step(mesh, gas, qm, cfg.dt, steps=1, work=work, opts=mixed)
        b.record()
        torch.cuda.synchronize()
        total_m += a.elapsed_time(b)
    if mesh.status() != 0:
        raise SystemExit("status flags set in the wall-bounded mixed-form run")
    ms_m = total_m / steps
    nbnd = int((case["face_bc"] != 0).sum())
    cpu = None
    if not args.no_cpu_baseline:  # the oracle's right-hand side on the channel at 6^3 x 6 tets (one core)
        import oracle.boundary as bd
        from oracle.geometry import connect, geometric_factors
        from oracle.refelem import build_reference
        from oracle.thermo import PerfectGas
        small = build_case(cfg, n=6)
        ref = build_reference(cfg.N, small["ref_nodes"])
        geo = geometric_factors(small["vertices"])
        conn = connect(small["vertices"], small["period"], ref, face_bc=small["face_bc"])
        t0 = time.perf_counter()
        bd.rhs_ns_bc(ref, geo, conn, small["q"], PerfectGas(g.gamma, g.R), g.mu, g.Pr)
        cpu_s = time.perf_counter() - t0
        cpu = {"value": small["q"].shape[1] * small["q"].shape[2] / cpu_s, "unit": "DOF-updates/s", "cores": 1, "host": host_cpu(),
               "sample": f"one right-hand side of the oracle on the channel at 6^3 x 6 tets, N = {cfg.N} "
                         f"(numpy, single thread), {cpu_s:.2f} s"}
    return {"workload": f"{cfg.name}: {cfg.description}", "K": cfg.K, "N": cfg.N, "Np": cfg.Np, "dtype": "f64",
            "boundary_faces": nbnd, "steps": steps, "ms_per_step": ms, "value": value, "unit": "DOF-updates/s",
            "vs_periodic_same_size": None if not periodic_fp64 else value / periodic_fp64,
            "kernels": kt,
            "mixed_form": {"ms_per_step": ms_m, "value": cfg.dofs * 5 / (ms_m * 1e-3), "unit": "DOF-updates/s",
                           "vs_fp64": ms / ms_m},
            "cpu_oracle_stage": cpu,
            "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


def av_form(args, local):
    """Shock capturing: Euler with artificial viscosity on two smoothed Sod fronts (24^3 x 6 tets,
    N = 3), FP64 RK4 steps with CUDA events and the kernel split, against the same steps with
    the artificial viscosity off; and the same steps in the mixed-precision form, with their state
    error against the FP64 form."""
    import numpy as np
    import torch
    from paper_2512_17101_gb300 import dg
    from workloads.configs import build_case, get_config

    cfg = get_config("euler_shock_av")
    dev = torch.device("cuda", local)
    case = build_case(cfg)
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"])
    gas = dg.Gas(model="perfect", gamma=cfg.gas.gamma, R=cfg.gas.R)
    q0 = torch.tensor(case["q"], device=dev)
    work = (torch.empty_like(q0), torch.zeros_like(q0))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    params = dict(eps0=5e-3, s0=-4.0 * np.log10(cfg.N), kappa=1.0)

    from paper_2512_17101_gb300 import capi
    mixed = dg._opts(precision=capi.DG_PREC_MIXED)

    def run(on, opts=None):
        mesh.set_av(params["eps0"] if on else 0.0, params["s0"], params["kappa"])
        q = q0.clone()
        for _ in range(max(3, args.warmup)):
            dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, work=work, opts=opts)
        q.copy_(q0)
        mesh.kernel_times(reset=True)
        mesh.set_timing(True)
        total = 0.0
        for _ in range(max(1, args.steps)):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, work=work, opts=opts)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
        mesh.set_timing(False)
        kt = {n: {"avg_ms": ms / c, "launches": c} for n, (ms, c) in mesh.kernel_times(reset=True).items() if c}
        if mesh.status() != 0:
            raise SystemExit("status flags set in the artificial-viscosity run")
        return total / max(1, args.steps), kt, q

    ms_on, kt_on, q64 = run(True)
    ms_off, _, _ = run(False)
    ms_mx, kt_mx, qmx = run(True, mixed)
    a64, amx = q64.cpu().numpy(), qmx.cpu().numpy()
    groups = [[0], [1, 2, 3], [4]]
    mixed_err = max(max(np.abs(amx[v] - a64[v]).max() for v in g) / max(np.abs(a64[v]).max() for v in g)
                    for g in groups)
    mesh.set_av(params["eps0"], params["s0"], params["kappa"])
    eps = torch.empty(cfg.K, dtype=torch.float64, device=dev)
    mesh.av_viscosity(q0, eps)
    e = eps.cpu().numpy()
    return {"workload": f"{cfg.name}: {cfg.description}", "K": cfg.K, "N": cfg.N, "dtype": "f64",
            "steps": max(1, args.steps), "ms_per_step": ms_on, "value": cfg.dofs * 5 / (ms_on * 1e-3),
            "unit": "DOF-updates/s", "ms_per_step_without_av": ms_off, "av_overhead": ms_on / ms_off - 1.0,
            "kernels": kt_on, "elements_with_eps": {"zero": int((e == 0).sum()), "ramp": int(((e > 0) & (e < 5e-3)).sum()),
                                                      "eps0": int((e == 5e-3).sum())},
            "mixed": {"ms_per_step": ms_mx, "value": cfg.dofs * 5 / (ms_mx * 1e-3), "kernels": kt_mx,
                      "speedup_vs_fp64": ms_on / ms_mx,
                      "state_error_vs_fp64": {"per_field_max": mixed_err, "steps": max(1, args.steps),
                                              "fields": "rho, momentum as one vector, rho E"}},
            "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


def mixture_ns_form(args, local):
    """The viscous mixture with species diffusion (7 species, the mixture workload's mesh and
    state: 32^3 x 6 tets, N = 2), FP64 RK4 steps with CUDA events and the kernel split, against
    the same steps without viscosity."""
    import numpy as np
    import torch
    from paper_2512_17101_gb300 import dg
    from workloads.configs import build_case, get_config

    cfg = get_config("mixture_learned")
    dev = torch.device("cuda", local)
    case = build_case(cfg)
    mix = case["mixture"]
    mesh = dg.Mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"])
    Rk = 8314.462618 / np.asarray(mix.W)
    Rmix = np.einsum("k,k...->...", Rk, case["Y"])
    rho = case["p0"] / (Rmix * case["T"])
    # conserved state from (rho, u, Y, T) with the library's own energy evaluation
    e = torch.empty(case["T"].size, dtype=torch.float64, device=dev)
    out = {}
    for visc in (True, False):
        gas = dg.Gas(model="nasa7", W=mix.W, nasa7=mix.coeffs, newton_tol=1e-10, newton_max_it=50,
                     mu=1.8e-5 if visc else 0.0, Pr=0.71, Sc=0.7)
        dg.dg_mixture_energy(gas, torch.tensor(np.ascontiguousarray(case["T"].ravel()), device=dev),
                             torch.tensor(np.ascontiguousarray(case["Y"].reshape(case["Y"].shape[0], -1)),
                                          device=dev).contiguous(), e)
        ee = e.cpu().numpy().reshape(case["T"].shape)
        vel = case["vel"]
        E = rho * (ee + 0.5 * np.sum(vel ** 2, axis=0))
        q0 = torch.tensor(np.concatenate([rho[None], rho[None] * vel, E[None], rho[None] * case["Y"]]), device=dev)
        q = q0.clone()
        T = torch.tensor(case["T"], device=dev)
        work = (torch.empty_like(q), torch.zeros_like(q))
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        for _ in range(max(3, args.warmup)):
            dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, T_io=T, work=work)
        q.copy_(q0)
        mesh.kernel_times(reset=True)
        mesh.set_timing(True)
        total = 0.0
        for _ in range(max(1, args.steps)):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dg.lsrk4_step(mesh, gas, q, cfg.dt, steps=1, T_io=T, work=work)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
        mesh.set_timing(False)
        kt = {n: {"avg_ms": ms / c, "launches": c} for n, (ms, c) in mesh.kernel_times(reset=True).items() if c}
        if mesh.status() != 0 or gas.status() != 0:
            raise SystemExit("status flags set in the viscous-mixture run")
        out[visc] = (total / max(1, args.steps), kt)
    ms, kt = out[True]
    return {"workload": f"{cfg.name} mesh and state with viscosity (mu = 1.8e-5, Pr = 0.71, Sc = 0.7): 7-species "
                        f"NASA-7 mixture, 32^3 x 6 = 196,608 tets, N = 2, species and enthalpy diffusion",
            "K": cfg.K, "N": cfg.N, "V": 12, "dtype": "f64", "steps": max(1, args.steps), "ms_per_step": ms,
            "value": cfg.dofs * 5 / (ms * 1e-3), "unit": "DOF-updates/s", "ms_per_step_inviscid": out[False][0],
            "kernels": kt, "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


def hex_advection_flops_per_element(M, velocity):
    """FP64 flops of the advection right-hand side + stage update per element (M = N+1): per node
    3 line derivatives of M FMAs (the factor -a_d (2/h_d) dt folded into D) and the 2 FMAs of the
    update; per node of an inflow face (one per axis with a_d != 0) a difference and an FMA."""
    inflow = sum(1 for v in velocity if v != 0.0)
    return M ** 3 * (2 * 3 * M + 2 * 2) + inflow * M * M * 3


def hex_shock_form(args, local):
    """Navier-Stokes with artificial viscosity and walls on p = 1 hexahedra, 256 x 128 x 32 box
    (1,048,576 hexahedra, 8.4 M DOFs): Mach 3 inflow at x = 0, outflow at x = 2, no-slip adiabatic
    walls at y = 0 and 1, periodic in z, a smoothed Sod front across x = 0.5.  Times the RK4
    stage and reports the right-hand-side throughput (DOFs per second per evaluation)."""
    import numpy as np
    import torch
    from paper_2512_17101_gb300 import capi, dg
    from workloads.hexmesh import gll_nodes, hex_box, hex_nodes

    dev = torch.device("cuda", local)
    n, N, L = (256, 128, 32), 1, (2.0, 1.0, 0.25)
    box = hex_box(n, L)
    x1 = gll_nodes(N)
    xyz = hex_nodes(box, x1)
    x = xyz[..., 0]
    S = 0.5 * (1.0 + np.tanh((0.5 - x) / 0.01))  # 1 upstream of the front, 0 downstream
    rho = 0.125 + 0.875 * S
    p = 0.1 + 0.9 * S
    u = 3.0 * np.sqrt(1.4) * S  # Mach 3 upstream (c = sqrt(1.4 p / rho) = sqrt(1.4))
    zero = np.zeros_like(x)
    E = p / 0.4 + 0.5 * rho * u * u
    q_host = np.stack([rho, rho * u, zero, zero, E])
    bc = ((capi.DG_BC_INFLOW, capi.DG_BC_OUTFLOW), (capi.DG_BC_NOSLIP_WALL, capi.DG_BC_NOSLIP_WALL), (0, 0))
    mesh = dg.HexMesh(box["n"], box["L"], N, x1, bc=bc)
    mesh.set_inflow(q_host[:, 0, 0])
    mesh.set_av(5e-3, -4.0 * np.log10(max(N, 2)), 1.0)
    gas = dg.Gas(model="perfect", gamma=1.4, R=1.0, mu=1e-4, Pr=0.71)
    q0 = torch.tensor(q_host, device=dev)
    K, Np = mesh.K, mesh.Np
    dt = 0.3 * (L[0] / n[0]) / ((N + 1) ** 2 * (3.0 * np.sqrt(1.4) + np.sqrt(1.4)))
    q = q0.clone()
    work = (torch.empty_like(q), torch.zeros_like(q))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        dg.hex_lsrk4_step(mesh, gas, q, dt, steps=1, work=work)
    q.copy_(q0)
    steps = max(1, args.steps)
    total = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.hex_lsrk4_step(mesh, gas, q, dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    if mesh.status() != 0:
        raise SystemExit("status flags set in the hexahedral shock run")
    eps = torch.empty(K, dtype=torch.float64, device=dev)
    mesh.av_viscosity(q0, eps)
    ms = total / steps
    dofs = K * Np
    return {"workload": "p = 1 hexahedra, 256 x 128 x 32 box (8.4 M DOFs per field): Navier-Stokes "
                        "(mu = 1e-4, Pr = 0.71) with artificial viscosity (eps0 = 5e-3), Mach 3 inflow, "
                        "outflow, no-slip adiabatic walls, smoothed Sod front", "K": K, "N": N, "dtype": "f64",
            "steps": steps, "ms_per_step": ms, "value": dofs * 5 / (ms * 1e-3), "unit": "DOF-updates/s",
            "elements_with_eps": int((eps > 0).sum().item()),
            "context": "the paper quotes 100.4 M DOFs/s of right-hand-side throughput on one MI300A for its "
                       "p = 1 tensor-product shock/boundary-layer case (2-D); this 3-D analogue's figure is "
                       "the same quantity (DOFs x RHS evaluations per second), not a like-for-like target",
            "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


def hex_advection_form(args, local):
    """Scalar advection on p = 1 hexahedra (the paper's GPU comparison workload), 128^3 hexahedra:
    FP64 RK4 steps with CUDA events, the FP64 and HBM rooflines, and the oracle's stage on 32^3."""
    import torch
    from paper_2512_17101_gb300 import dg
    from workloads.configs import build_hex_advection_case, get_config

    cfg = get_config("hex_advection")
    dev = torch.device("cuda", local)
    case = build_hex_advection_case(cfg)
    vel = case["velocity"]
    mesh = dg.HexMesh(case["box"]["n"], case["box"]["L"], cfg.N, case["nodes1d"])
    u0 = torch.tensor(case["u"], device=dev)
    u = u0.clone()
    work = (torch.empty_like(u), torch.zeros_like(u))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        dg.hex_advection_lsrk4_step(mesh, vel, u, cfg.dt, steps=1, work=work)
    u.copy_(u0)
    steps = max(1, args.steps)
    total = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.hex_advection_lsrk4_step(mesh, vel, u, cfg.dt, steps=1, work=work)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    ms = total / steps
    M = cfg.N + 1
    stage_s = ms * 1e-3 / 5
    flops = hex_advection_flops_per_element(M, vel) * cfg.K
    nbytes = M ** 3 * 8 * 4 * cfg.K  # u in, k in and out, u_out
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    cpu = None
    if not args.no_cpu_baseline:  # the oracle's stage on a 32^3 box (one core), for context
        import oracle.hex as hx
        small = build_hex_advection_case(cfg, n=32)
        ref = hx.hex_reference(small["nodes1d"])
        t0 = time.perf_counter()
        hx.hex_advection_rhs_strong(ref, small["box"], small["u"], vel)
        cpu_s = time.perf_counter() - t0
        cpu = {"value": 32 ** 3 * M ** 3 / cpu_s, "unit": "DOF-updates/s", "cores": 1, "host": host_cpu(),
               "sample": f"one right-hand side of the oracle on 32^3 hexahedra, N = {cfg.N} "
                         f"(numpy, single thread), {cpu_s:.2f} s"}
    return {"workload": f"{cfg.name}: {cfg.description}", "K": cfg.K, "N": cfg.N, "Np": M ** 3, "dtype": "f64",
            "steps": steps, "ms_per_step": ms, "value": cfg.dofs * 5 / (ms * 1e-3), "unit": "DOF-updates/s",
            "roofline": {"bound": "alu", "achieved": flops / stage_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / stage_s / 1e12 / FP64_PEAK_TFLOPS,
                         "flops_per_stage": flops, "algorithmic_bytes_per_stage": nbytes,
                         "hbm_achieved_gbs": nbytes / stage_s / 1e9, "hbm_frac": nbytes / stage_s / 1e9 / hbm},
            "cpu_oracle_stage": cpu,
            "l2": "256 MiB buffer written before every timed step (outside the step's events)"}


def partitioned_form(args, local, whole_ms=None):
    """The Navier-Stokes workload (24^3 x 6 tets, N = 3) split into two element partitions (z
    slabs, each with its halo) held on one device: every stage refreshes the halos of the state and
    of the BR1 viscous flux through the library's gather / scatter kernels, handed over by the
    in-process router (between GPUs the same buffers would travel as torch.distributed
    point-to-point messages), with each partition's interior elements computed between posting an
    exchange and finishing it and its border elements after.  RK4 steps with CUDA events against
    the same steps on the whole mesh; owned DOFs only count toward the value."""
    import numpy as np
    import torch
    from paper_2512_17101_gb300 import dg
    from paper_2512_17101_gb300.partition import (HaloExchange, LocalRouter, RankState, partition_mesh,
                                                  partitioned_lsrk4_step)
    from workloads.configs import build_case, get_config

    cfg = get_config("ns_viscous")
    dev = torch.device("cuda", local)
    case = build_case(cfg)
    g = cfg.gas
    gas = dg.Gas(model="perfect", gamma=g.gamma, R=g.R, mu=g.mu, Pr=g.Pr)
    parts = partition_mesh(case["vertices"], case["period"], cfg.N, case["ref_nodes"], 2)
    ranks = []
    for p in parts:
        m = dg.Mesh(p.vertices, case["period"], cfg.N, case["ref_nodes"], face_bc=p.face_bc)
        q = torch.tensor(np.ascontiguousarray(case["q"][:, p.local]), device=dev)
        ranks.append(RankState(m, HaloExchange(p, m.Np, dev), q, (torch.empty_like(q), torch.zeros_like(q))))
    q0 = [r.q.clone() for r in ranks]
    router = LocalRouter()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        partitioned_lsrk4_step(ranks, gas, router, cfg.dt)
    for r, q in zip(ranks, q0):
        r.q.copy_(q)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        partitioned_lsrk4_step(ranks, gas, router, cfg.dt)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    for r in ranks:
        if r.mesh.status() != 0:
            raise SystemExit("status flags set in the partitioned run")
    ms = total / max(1, args.steps)
    halo = sum(len(p.halo) for p in parts)
    per_stage = sum(len(ix) for p in parts for ix in p.recv.values()) * cfg.Np * 8 * (5 + (9 if g.mu > 0 else 0))
    out = {"workload": f"{cfg.name} in 2 partitions on one device: {cfg.description}", "K": cfg.K, "N": cfg.N,
           "dtype": "f64", "steps": max(1, args.steps), "ms_per_step": ms,
           "value": cfg.dofs * 5 / (ms * 1e-3), "unit": "DOF-updates/s (owned DOFs)",
           "halo_elements": halo, "halo_fraction": halo / cfg.K,
           "interior_elements": sum(p.n_interior for p in parts),
           "schedule": "per stage: post the state's exchange; owned primitives, interior viscous flux; finish; "
                       "halo primitives, border viscous flux; post the flux's exchange; interior stages; finish; "
                       "border stages (interior work overlaps each exchange between GPUs)",
           "exchange_bytes_per_step": 5 * per_stage,
           "transport": "in-process router (no copy); the bytes are what each stage moves between partitions",
           "l2": "256 MiB buffer written before every timed step (outside the step's events)"}
    if whole_ms:
        out["ms_per_step_whole_mesh"] = whole_ms
        out["overhead"] = ms / whole_ms - 1.0
    return out


def batched_form(args, local):
    """The batched workload (64 uneven cases, orders 1..4, half Euler / half NS, mixed precision):
    one graph launch per RK4 step, against stepping the same cases one by one."""
    import torch
    from paper_2512_17101_gb300 import capi, dg
    from workloads.configs import batched_cases

    dev = torch.device("cuda", local)
    cases = batched_cases(64, seed=0)
    hs = []
    for c in cases:
        mesh = dg.Mesh(c["vertices"], c["period"], c["N"], c["ref_nodes"])
        g = c["gas"]
        gas = dg.Gas(model="perfect", gamma=g.gamma, R=g.R, mu=g.mu, Pr=g.Pr)
        hs.append((mesh, gas, c["dt"], torch.tensor(c["q"], device=dev)))
    t0 = time.perf_counter()
    batch = dg.Batch(hs, autotune=True)
    setup_s = time.perf_counter() - t0
    dofs = sum(c["K"] * c["Np"] for c in cases)
    steps = max(2, min(args.steps, 10))
    batch.step(2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    batch.step(steps)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    if batch.status() != 0:
        raise SystemExit("status flags set in the batched run")
    # the same cases stepped one by one (one call per case and stage)
    opts = dg._opts(precision=capi.DG_PREC_MIXED)
    works = [(torch.empty_like(q), torch.zeros_like(q)) for (_, _, _, q) in hs]
    for (mesh, gas, dt, q), w in zip(hs, works):
        dg.lsrk4_step(mesh, gas, q, dt, steps=1, opts=opts, work=w)
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        for (mesh, gas, dt, q), w in zip(hs, works):
            dg.lsrk4_step(mesh, gas, q, dt, steps=1, opts=opts, work=w)
    b.record()
    torch.cuda.synchronize()
    ms_seq = a.elapsed_time(b) / steps
    rt, vt, tune = batch.tiles()
    # algorithmic bytes of one graph launch (RK4 step): per stage and case the primitives pass, the
    # BR1 pass of a viscous case and the right-hand side with its RK update; then the copy of each
    # case's result back into its state (read + write of the FP64 state)
    step_bytes = 0
    for c in cases:
        Np, NF, visc = c["Np"], 4 * (c["N"] + 1) * (c["N"] + 2) // 2, c["gas"].mu > 0
        per_el = mixed_prims_bytes_per_element(Np, visc) + mixed_rhs_bytes_per_element(Np, NF, visc)
        if visc:
            per_el += mixed_viscous_bytes_per_element(Np, NF)
        step_bytes += c["K"] * (5 * per_el + 2 * 5 * 8 * Np)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)  # the recipe's fallback when the file is absent
    achieved = step_bytes / (ms * 1e-3) / 1e9
    return {"workload": "64 cases, periodic n^3 x 6 tets with n ~ U{2..20}, N ~ U{1..4}, half Euler vortex / half "
                        "NS Taylor-Green, seed 0; mixed precision",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "algorithmic_bytes_per_step": step_bytes,
                         "note": "whole graph launch (all kernels and the copies), measured copy peak"},
            "dofs_per_stage": dofs, "steps": steps, "ms_per_step": ms, "value": dofs * 5 / (ms * 1e-3),
            "unit": "DOF-updates/s", "graph_launches_per_step": 1, "setup_s_incl_autotune": setup_s,
            "one_by_one_ms_per_step": ms_seq, "one_by_one_value": dofs * 5 / (ms_seq * 1e-3),
            "tiles_rhs_by_order_euler_ns": rt.tolist(), "tiles_br1_by_order": vt.tolist()}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--config", default="ns_viscous")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form section")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form section")
    ap.add_argument("--no-hex", action="store_true", help="skip the tensor-product hexahedron section")
    ap.add_argument("--no-overint", action="store_true", help="skip the over-integration section")
    ap.add_argument("--no-boundary", action="store_true", help="skip the wall-bounded channel, artificial-viscosity and viscous-mixture sections")
    ap.add_argument("--no-partitioned", action="store_true", help="skip the two-partition section")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="form timed for the headline value (the other form is reported beside it)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    from workloads.configs import get_config
    cfg = get_config(args.config)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        reference_arm(args, cfg, world, rank)
    else:
        gpu_arm(args, cfg, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
