#!/usr/bin/env python
"""Benchmark of the spectral/hp Helmholtz operator on GB300.

A step is one application of the Helmholtz operator H = lambda M + L (BwdTrans,
reference gradient, pointwise geometric factors, transposed gradient and
IProductWRTBase fused in one kernel launch) to every element of the workload
mesh: by default 32^3 curved hexes, P = 4, Q = 6, the operator applied in FP64
(the arithmetic of the workload), which on this part is bound by the FP64 pipe:
its roofline divides by the FP64 peak measured in the same run by the probe
kernels of csrc/peak_probe.cu.  The FP32 apply of the same workload (bound by
HBM) is reported under "f32" with its own roofline and end-to-end figure.
Prints one JSON line.

Besides the timed steps it reports, each measured separately after the timed
region and each with its roofline: PhysDeriv, BwdTrans, IProduct, FwdTrans,
Integral (both precisions) and the sensor, the variable-order workload (24^3
hexes, P_e in 2..8), the adjoint workload (16^3 hexes, P = 6) and the periodic
solve of the 48^3 workload to a 1e-10 relative residual in FP32-inner + FP64
refinement (restarted, and with reliable updates) and in all-FP64 CG.

Multi-GPU (torchrun, one rank per GPU): every rank applies the operator to
its own copy of the workload (independent element partitions, no exchange):
weak scaling; value = all ranks' DOFs / max-over-ranks time.

--impl reference times the FP64 CPU oracle (dense elemental matrices) on a
bounded sample of the same workload on the host cores.
"""
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

METRIC = "Helmholtz apply GDOF/s and % HBM roofline; CG time-to-1e-10 FP32+refine vs FP64"
L2_BYTES = 129 * 1024 * 1024


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 ALU peak derived from unit counts and the maximum SM clock: 152 SMs x
# 2 FP64 FMA per clock x 2 flop x 2.07 GHz.  Reported beside the measured
# peak (fp_peaks) for context; the roofline divides by the measured one.
FP64_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def helm_bytes_per_elem(P, Q, sz, dim=3):
    n = P + 1
    return (2 * n ** dim + (7 if dim == 3 else 4) * Q ** dim) * sz


def helm_flops_per_elem(P, Q):
    """Algorithmic flops of one element's Helmholtz apply (direct 1D contractions)."""
    n = P + 1
    bwd = n ** 3 * Q + n ** 2 * Q ** 2 + n * Q ** 3
    return 2 * (2 * bwd + 6 * Q ** 4) + 20 * Q ** 3


def _eo_ops(P, Q):
    """(flops, FP64 instructions) of the even-odd 1D contractions of the
    Helmholtz bodies: B and dB (n -> Q), B^T (Q -> n) and D / D^T (Q -> Q).
    A product started from zero is one multiply (1 flop), every other term
    one FMA (2 flops); the sums and differences of the even-odd split are
    adds."""
    H, Hc = Q // 2, (Q + 1) // 2
    nodd = len([b for b in range(1, P) if b % 2])
    nev = len([b for b in range(2, P) if b % 2 == 0])
    b = (2 + Hc * (1 + 2 * nodd) + H * (3 + 2 * nev), 2 + Hc * (1 + nodd) + H * (3 + nev))
    db = (2 + Hc * (1 + 2 * nev) + H * (3 + 2 * nodd), 2 + Hc * (1 + nev) + H * (3 + nodd))
    bt_f, bt_i = 2 * H + (2 * Hc - 1) + (2 * H - 1) + 2, 2 * H + Hc + H + 2
    for k in range(1, P):
        m = Hc if k % 2 else H
        bt_f, bt_i = bt_f + 2 * m - 1, bt_i + m
    odd = Q % 2
    d = (2 * H + H * (4 * H + 2 * odd) + odd * (2 * H - 1), 2 * H + H * (2 * H + odd + 2) + odd * H)
    return b, db, (bt_f, bt_i), d


def helm_executed_ops_per_elem(P, Q):
    """(flops, FP64 instructions) the 3D Helmholtz body executes per element
    (no kappa field, constant lambda): B along xi_1, xi_2 on n^2 and n Q
    pencils and along xi_3 on Q^2 columns, where dB also gives the xi_3
    gradient; D along xi_1, xi_2 and D^T along all three directions on Q^2
    pencils / columns; per quadrature point 3 multiplies and 6 FMAs for
    G grad u, one multiply for lambda JW, one FMA adding the mass term and two
    adds joining the three transposed-gradient parts; B^T back to the modes
    on Q^2, n Q and n^2 pencils."""
    n = P + 1
    b, db, bt, d = _eo_ops(P, Q)
    terms = [(n * n + n * Q + Q * Q, b), (Q * Q, db), (5 * Q * Q, d), (Q * Q + n * Q + n * n, bt)]
    fl = sum(k * x[0] for k, x in terms) + Q ** 3 * (15 + 1 + 2 + 2)
    ins = sum(k * x[1] for k, x in terms) + Q ** 3 * (9 + 1 + 1 + 2)
    return fl, ins


def fp_peaks(torch, sampler_index=0):
    """Arithmetic peaks measured on this GPU by the committed probe kernels
    (csrc/peak_probe.cu): TFLOP/s of DFMA, DMMA (m8n8k4, m16n8k16), FFMA and
    FFMA2, each timed with CUDA events after a warm-up launch, the SM clock
    sampled meanwhile; plus the DFMA/DMMA sharing test."""
    import ctypes as C
    lib = C.CDLL(os.path.join(ROOT, "paper_1906_03489_gb300", "lib", "libspx_probe.so"))
    f = lib.spx_probe_rate
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)]
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    iters = {0: 1200, 1: 150, 2: 150, 3: 60000, 4: 30000, 5: 400}
    names = {0: "dfma", 1: "dmma_m8n8k4", 2: "dmma_m16n8k16", 3: "ffma", 4: "ffma2", 5: "dfma_dmma_mixed"}
    out, raw = {}, {}
    with ClockSampler(sampler_index) as clk:
        for k in range(6):
            fl, ms = C.c_double(), C.c_float()
            rc = f(k, 4, max(1, iters[k] // 10), st, C.byref(fl), C.byref(ms))     # warm-up
            if rc == 0:
                rc = f(k, 4, iters[k], st, C.byref(fl), C.byref(ms))
            if rc != 0:
                out[names[k]] = {"error": rc}
                continue
            raw[k] = (fl.value, ms.value * 1e-3)
            out[names[k]] = round(fl.value / (ms.value * 1e-3) / 1e12, 4)
    if all(k in raw for k in (0, 1, 5)):
        # the mixed launch: its DFMA half and its DMMA half at the rates measured alone
        fl5, t5 = raw[5]
        fl_f = fl5 * 64 / (64 + 512)
        t_f = fl_f / (raw[0][0] / raw[0][1])
        t_m = (fl5 - fl_f) / (raw[1][0] / raw[1][1])
        out["dfma_dmma_mixed_s"] = {"measured": round(t5, 5), "if_one_unit": round(t_f + t_m, 5),
                                    "if_separate_units": round(max(t_f, t_m), 5)}
    fp64 = [out[n] for n in ("dfma", "dmma_m8n8k4", "dmma_m16n8k16") if isinstance(out.get(n), float)]
    out["fp64_peak_tflops"] = max(fp64) if fp64 else None
    out["clocks"] = clk.summary()
    out["how"] = ("probe kernels of csrc/peak_probe.cu, 4 blocks x 256 threads per SM, 8 independent chains per "
                  "thread, CUDA events; fp64_peak = the fastest FP64 kind")
    return out


# Sources of the Helmholtz kernels and their launcher (what their ncu counters depend on):
# the FP32 pair kernel (helm_pair.cuh and what it builds on) and the FP64 role body.
HELM_SOURCES = ("helm_pair.cuh", "op_kernel.cuh", "lanes.cuh", "kernel_params.h", "device_common.cuh",
                "launch_ops.cuh", "smem_layout.h")
HELM64_SOURCES = ("op_kernel.cuh", "lanes.cuh", "kernel_params.h", "device_common.cuh", "launch_ops.cuh",
                  "smem_layout.h")


def kernel_digest(names=None):
    """Digest of the library sources (all of them, or the named files of csrc/)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1906_03489_gb300", "csrc")
    if names is None:
        files = [(d, n) for d in (csrc, os.path.join(ROOT, "include")) for n in sorted(os.listdir(d))]
    else:
        files = [(csrc, n) for n in names]
    for d, name in files:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(name, sources=HELM_SOURCES):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_digest") == kernel_digest(sources):
            return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
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
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(name, spx, mesh, synth, torch, copies=1):
    w = synth.WORKLOADS[name]
    dim, N, amp = w["dim"], w["N"], w["amp"]
    E = N ** dim
    gen = synth.rng(w["seed"])
    if isinstance(w["P"], tuple):
        orders = synth.orders(gen, E, *w["P"])
        plans = [spx.Plan(dim, E, orders=orders) for _ in range(copies)]
        node_orders = orders
    else:
        plans = [spx.Plan(dim, E, order=w["P"]) for _ in range(copies)]
        node_orders = w["P"]
    nodes = mesh.structured_nodes(dim, N, node_orders, amp)
    geoms = []
    for p in plans:
        g = spx.geom_factors(p, nodes)
        p.set_geometry(torch.float64, g["geom"], g["dxi"])
        p.set_geometry(torch.float32, g["geom32"], g["dxi32"])
        geoms.append(g)
    coef = synth.uniform(gen, plans[0].n_coef)
    return w, plans, geoms, coef


def timed(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def timed_rotating(torch, call, k, launches, stream):
    """Mean device time of one launch of a streaming operator: `call(i)` runs
    it on buffer copy i of k (inputs, outputs and the geometric factors it
    reads; k copies hold over twice the L2, so no launch finds its operands
    there).  The k calls are captured once in a CUDA graph and the graph is
    replayed between CUDA events on `stream`, so host time between launches
    is not counted."""
    for i in range(k):   # warm-up: launch tiles built before the capture
        call(i)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        for i in range(k):
            call(i)
    rounds = max(2, -(-launches // k))
    with torch.cuda.stream(stream):
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(rounds):
            g.replay()
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / (rounds * k)


def apply_steps(spx, torch, plans, ins, outs, steps, stream, local):
    """Times `steps` Helmholtz applies alternating between the two copies of
    the workload (inputs of both copies exceed the L2), CUDA events on the
    launching stream, the SM clock sampled meanwhile."""
    def step(i):
        k = i & 1
        spx.helmholtz(plans[k], ins[k], lam=1.0, out=outs[k])
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            step(i)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, clk.summary()


def e2e_pipeline(spx, torch, plan, coef, dt, k_e2e):
    """The apply end to end through the public API with host buffers: every
    step copies its input from pinned host memory, applies the operator and
    copies the result back.  Served as a pipeline on three streams with two
    device buffers each: the upload of step i+1 and the download of step i-1
    run on the copy engines while step i computes.  Returns (ms per step,
    bytes up, bytes down per step)."""
    uh = torch.tensor(coef, dtype=dt).pin_memory()
    yh = [torch.empty(plan.n_coef, dtype=dt).pin_memory() for _ in range(2)]
    ud = [torch.empty(plan.n_coef, dtype=dt, device="cuda") for _ in range(2)]
    yd = [torch.empty_like(ud[0]) for _ in range(2)]
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for k in range(2):   # every buffer starts free
        ev_comp[k].record(s_comp)
        ev_out[k].record(s_out)

    def e2e_step(i):
        k = i & 1
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_comp[k])          # ud[k] no longer read by step i-2
            ud[k].copy_(uh, non_blocking=True)
            ev_in[k].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(ev_in[k])
            s_comp.wait_event(ev_out[k])         # yd[k] downloaded by step i-2
            spx.helmholtz(plan, ud[k], lam=1.0, out=yd[k])
            ev_comp[k].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[k])
            yh[k].copy_(yd[k], non_blocking=True)
            ev_out[k].record(s_out)

    for i in range(4):
        e2e_step(i)
    torch.cuda.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(s_in)
    for i in range(k_e2e):
        e2e_step(i)
    t1e.record(s_out)          # after the last download, which follows every earlier step
    t1e.synchronize()
    torch.cuda.synchronize()
    nb = uh.numel() * uh.element_size()
    return t0e.elapsed_time(t1e) / k_e2e, nb, nb


def tune_pair(plans, dtype, ins, outs, P, tile):
    if tile:
        eb, nt, st = (int(x) for x in tile.split(","))
        for p in plans:
            p.set_tile("helmholtz", dtype, eb, nt, st)
    else:
        plans[0].autotune("helmholtz", dtype, ins[0], outs[0], reps=5)
        t = plans[0].get_tile("helmholtz", dtype, P)
        plans[1].set_tile("helmholtz", dtype, *t)
    return plans[0].get_tile("helmholtz", dtype, P)


def run_ours(a):
    import torch
    import paper_1906_03489_gb300 as spx
    from paper_1906_03489_gb300 import mesh, synth

    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (there is no CPU path)")
    spx.lib()
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    name = a.workload
    w, plans, geoms, coef = make_workload(name, spx, mesh, synth, torch, copies=2)
    P, Q = w["P"], w["P"] + 2
    E = plans[0].E
    dofs = E * (P + 1) ** 3
    # arithmetic peaks of this GPU (the FP64 roof of the headline)
    fpk = fp_peaks(torch, local)
    fp64_peak = fpk["fp64_peak_tflops"]

    # ---- headline: the FP64 apply (FP64 pipe bound on this part) ----------
    u64 = [torch.tensor(coef, device="cuda", dtype=torch.float64) for _ in plans]
    o64 = [torch.empty_like(x) for x in u64]
    tile64 = tune_pair(plans, torch.float64, u64, o64, P, a.tile64)
    for i in range(a.warmup):
        spx.helmholtz(plans[i & 1], u64[i & 1], lam=1.0, out=o64[i & 1])
    torch.cuda.synchronize()
    barrier(world)
    ms, clk = apply_steps(spx, torch, plans, u64, o64, a.steps, stream, local)
    barrier(world)
    ms = max_over_ranks(ms, world)
    value = world * dofs / (ms * 1e-3) / 1e9
    fl_launch = E * helm_flops_per_elem(P, Q)
    ex_fl, ex_ins = helm_executed_ops_per_elem(P, Q)
    bytes64 = E * helm_bytes_per_elem(P, Q, 8)
    achieved = fl_launch / (ms * 1e-3) / 1e12
    ms_e2e, up, down = e2e_pipeline(spx, torch, plans[0], coef, torch.float64, max(10, a.steps // 2))
    ms_e2e = max_over_ranks(ms_e2e, world)

    # ---- the FP32 apply (HBM bound) ---------------------------------------
    u32 = [torch.tensor(coef, device="cuda", dtype=torch.float32) for _ in plans]
    o32 = [torch.empty_like(x) for x in u32]
    tile32 = tune_pair(plans, torch.float32, u32, o32, P, a.tile)
    k32 = max(a.steps, 200)
    for i in range(max(a.warmup, 20)):
        spx.helmholtz(plans[i & 1], u32[i & 1], lam=1.0, out=o32[i & 1])
    torch.cuda.synchronize()
    barrier(world)
    ms32, clk32 = apply_steps(spx, torch, plans, u32, o32, k32, stream, local)
    barrier(world)
    ms32 = max_over_ranks(ms32, world)
    bytes32 = E * helm_bytes_per_elem(P, Q, 4)
    ach32 = bytes32 / (ms32 * 1e-3) / 1e9
    ms32_e2e, up32, down32 = e2e_pipeline(spx, torch, plans[0], coef, torch.float32, max(10, k32 // 10))
    ms32_e2e = max_over_ranks(ms32_e2e, world)

    extras = {}
    if a.extras and rank == 0:
        extras = measure_extras(spx, mesh, synth, torch, plans, geoms, coef, stream, hbm_peak, fp64_peak,
                                fpk.get("ffma2") if isinstance(fpk.get("ffma2"), float) else None)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(name, seconds=a.cpu_seconds)
    if rank == 0:
        mesh_desc = f"{w['N']}^3 curved hexes (x'=x+{w['amp']} sin2piy sin2piz)"
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GDOF/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "mesh": mesh_desc, "P": P, "Q": Q, "elements_per_gpu": E,
                       "local_dofs_per_gpu": dofs,
                       "op": "Helmholtz H=lambda M+L, lambda=1, unassembled, FP64 (FP64 FMA, FP64 accumulation)",
                       "tile_eb_threads_stages": list(tile64),
                       "l2": f"inputs {2 * bytes64 / 1e6:.0f} MB per step pair alternate between two "
                             f"independent copies (> {L2_BYTES / 1e6:.0f} MB L2): no L2 flush",
                       "parallelism": f"replica per GPU x{world}"},
            "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": round(achieved / fp64_peak, 4) if fp64_peak else None,
                         "traffic": profiled_traffic("helmholtz_f64_hex32.txt", HELM64_SOURCES),
                         "peak_kind": "measured: fastest FP64 probe kind on this GPU in this run (fp_peaks)",
                         "algorithmic_flops_per_launch": fl_launch,
                         "flops_model": "per element 2 (2 (n^3 Q + n^2 Q^2 + n Q^3) + 6 Q^4) + 20 Q^3 "
                                        "(direct 1D contractions, collocation gradient)",
                         "executed": {"flops_per_launch": E * ex_fl, "fp64_instructions_per_launch": E * ex_ins,
                                      "tflops": round(E * ex_fl / (ms * 1e-3) / 1e12, 4),
                                      "fp64_pipe_frac": round(2 * E * ex_ins / (ms * 1e-3) / 1e12 / fp64_peak, 4)
                                      if fp64_peak else None,
                                      "note": "even-odd contractions: fewer flops than the algorithmic count; "
                                              "fp64_pipe_frac counts every FP64 instruction (add, mul, fma) as "
                                              "one pipe slot of the DFMA rate"},
                         "derived_peak_tflops": round(FP64_DERIVED_TFLOPS, 4),
                         "hbm_frac": round(bytes64 / (ms * 1e-3) / 1e9 / hbm_peak, 4)},
            "e2e": {"value": round(world * dofs / (ms_e2e * 1e-3) / 1e9, 4), "unit": "GDOF/s",
                    "h2d_bytes_per_step": int(up), "d2h_bytes_per_step": int(down), "ms_per_step": round(ms_e2e, 4),
                    "steps": max(10, a.steps // 2),
                    "pipeline": "pinned host buffers; 3 streams, 2 device buffers each: the upload of step i+1 "
                                "and the download of step i-1 overlap the apply of step i"},
            "gpu_launches": a.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
            "f32": {
                "value": round(world * dofs / (ms32 * 1e-3) / 1e9, 4), "unit": "GDOF/s", "steps": k32,
                "ms_per_step": round(ms32, 5), "dtype": "f32",
                "op": "Helmholtz H=lambda M+L, lambda=1, unassembled, FP32 FMA/FP32 accumulate",
                "tile_eb_threads_stages": list(tile32),
                "roofline": {"bound": "hbm", "achieved": round(ach32, 1), "peak": hbm_peak, "unit": "GB/s",
                             "frac": round(ach32 / hbm_peak, 4), "traffic": profiled_traffic("helmholtz_f32_hex32.txt"),
                             "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes32,
                             "bytes_model": "per element (2 (P+1)^3 coefficients + 7 Q^3 geometric factors) x 4 B"},
                "e2e": {"value": round(world * dofs / (ms32_e2e * 1e-3) / 1e9, 4), "unit": "GDOF/s",
                        "h2d_bytes_per_step": int(up32), "d2h_bytes_per_step": int(down32),
                        "ms_per_step": round(ms32_e2e, 4), "steps": max(10, k32 // 10)},
                "clocks": clk32},
            "fp_peaks": fpk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def op_flops_per_elem(op, P, Q):
    """Algorithmic flops per 3D element of the operators besides Helmholtz
    (direct 1D contractions, as the generic kernel executes them)."""
    n = P + 1
    bwd = 2 * (n ** 3 * Q + n ** 2 * Q ** 2 + n * Q ** 3)
    mass = 2 * bwd + Q ** 3                      # BwdTrans, JW, IProduct
    pre = 3 * 2 * n ** 4                         # (M1^-1) along three directions
    return {"bwd_trans": bwd, "iproduct": bwd + Q ** 3, "phys_deriv": 6 * Q ** 4 + 18 * Q ** 3,
            "integral": 2 * Q ** 3,
            # b = IProduct(f), z = K^-1 b, then one PCG step (the preconditioner is exact where det J is
            # constant on the element, as on this mesh): M p, K^-1 r, and ~12 n^3 of vector work
            "fwd_trans": (bwd + Q ** 3) + 2 * pre + mass + 12 * n ** 3,
            # u^T M u, one restricted PCG step as above, then d^T M d
            "sensor": 3 * mass + 2 * pre + 14 * n ** 3}[op]


def roof(ms, nbytes, nflops, fp64, hbm_peak, fp_peak):
    """Roofline figures of one launch: HBM and ALU fractions; `bound` is the
    FP64 pipe for FP64 kernels (machine balance about 0.2 flop/B), HBM for FP32."""
    gbs = nbytes / ms / 1e6
    tfl = nflops / ms / 1e9
    r = {"ms": round(ms, 4), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
         "tflops": round(tfl, 4), "algorithmic_bytes": int(nbytes), "algorithmic_flops": int(nflops)}
    if fp_peak:
        r["alu_frac"] = round(tfl / fp_peak, 4)
    r["bound"] = "alu" if fp64 else "hbm"
    r["frac"] = r.get("alu_frac") if fp64 else r["hbm_frac"]
    return r


def measure_extras(spx, mesh, synth, torch, plans, geoms, coef, stream, hbm_peak, fp64_peak, fp32_peak=None):
    """Other operators / precisions / workloads, each timed after warm-up with
    CUDA events, each with its roofline: FP64 kernels against the measured
    FP64 peak (ALU), FP32 kernels against the HBM peak (their ALU fraction
    against the measured FFMA peak beside it)."""
    ex = {}
    plan = plans[0]
    P, Q, E = 4, 6, plan.E
    n3 = (P + 1) ** 3
    reps = 30
    ops = {}
    geo0 = geoms[0]
    for dt, sz in ((torch.float32, 4), (torch.float64, 8)):
        fp64 = dt == torch.float64
        pk = fp64_peak if fp64 else fp32_peak
        gk = ("geom", "dxi") if fp64 else ("geom32", "dxi32")
        c = torch.tensor(coef, device="cuda", dtype=dt)
        f = spx.bwd_trans(plan, c)
        tag = "f32" if dt == torch.float32 else "f64"
        # streaming operators, each over k copies of its operands (> 2 x L2 in all)
        for op, nbytes, nq_out in (("phys_deriv", E * 13 * Q ** 3 * sz, 3), ("bwd_trans", E * (n3 + Q ** 3) * sz, 1),
                                   ("iproduct", E * (2 * Q ** 3 + n3) * sz, 0)):
            k = max(2, -(-2 * L2_BYTES // nbytes))
            src = c if op == "bwd_trans" else f
            ins = [src.clone() for _ in range(k)]
            outs = [torch.empty(nq_out * plan.n_quad if nq_out else plan.n_coef, dtype=dt, device="cuda")
                    for _ in range(k)]
            geos = [(geo0[gk[0]].clone(), geo0[gk[1]].clone()) for _ in range(k)] if op != "bwd_trans" else None

            def call(i, op=op, ins=ins, outs=outs, geos=geos):
                if geos:
                    plan.set_geometry(dt, *geos[i])
                if op == "phys_deriv":
                    spx.phys_deriv(plan, ins[i], list(outs[i].view(3, -1)))
                elif op == "bwd_trans":
                    spx.bwd_trans(plan, ins[i], outs[i])
                else:
                    spx.iproduct(plan, ins[i], outs[i])
            if geos:
                plan.set_geometry(dt, *geos[0])
            plan.autotune(op, dt, ins[0], outs[0], reps=5)
            ms = timed_rotating(torch, call, k, 60, stream)
            plan.set_geometry(dt, geo0[gk[0]], geo0[gk[1]])
            r = roof(ms, nbytes, E * op_flops_per_elem(op, P, Q), fp64, hbm_peak, pk)
            r["tile_eb_threads_stages"] = list(plan.get_tile(op, dt, P))
            r["timing"] = (f"{k} copies of the operands ({k * nbytes / 1e6:.0f} MB, > 2 x L2) launched in turn "
                           "from a CUDA graph, CUDA events around the replays")
            ops[f"{op}_{tag}"] = r
            del ins, outs, geos
        # FwdTrans (elemental preconditioned CG in one launch; reads f and JW, writes the coefficients)
        # and Integral (reads f and JW)
        f = spx.bwd_trans(plan, torch.tensor(coef, device="cuda", dtype=dt))
        if fp64:   # FwdTrans is FP64 only (an FP32 projection cannot meet the FP32 bar: cond(M_e) > 2^24)
            cf = torch.empty(plan.n_coef, dtype=dt, device="cuda")
            plan.autotune("fwd_trans", dt, f, cf, reps=3)
            ms = timed(lambda: spx.fwd_trans(plan, f, cf), reps, stream)
            r = roof(ms, E * (2 * Q ** 3 + n3) * sz, E * op_flops_per_elem("fwd_trans", P, Q), fp64, hbm_peak, pk)
            r["tile_eb_threads_stages"] = list(plan.get_tile("fwd_trans", dt, P))
            r["max_err_vs_input_coefficients"] = (cf.double() - torch.tensor(coef, device="cuda")).abs().max().item()
            r["bound_on_that_error"] = "cond(M_e) x 2^-52 x |c| ~ 1e-8 (coefficients of a cond 4.5e7 system)"
            ops[f"fwd_trans_{tag}"] = r
        if fp64:   # adaptive-order sensor (FP64): reads the coefficients and JW, writes one value per element
            cc = torch.tensor(coef, device="cuda")
            so = torch.empty(plan.E, dtype=torch.float64, device="cuda")
            plan.autotune("sensor", dt, cc, so, reps=3)
            ms = timed(lambda: spx.sensor(plan, cc, so), reps, stream)
            ops["sensor_f64"] = roof(ms, E * (n3 + Q ** 3 + 1) * sz, E * op_flops_per_elem("sensor", P, Q), True,
                                     hbm_peak, pk)
            ops["sensor_f64"]["tile_eb_threads_stages"] = list(plan.get_tile("sensor", dt, P))
        # a reduction streaming 2 Q^3 values per element: HBM bound in both precisions
        nbytes = E * 2 * Q ** 3 * sz
        k = max(2, -(-2 * L2_BYTES // nbytes))
        ins = [f.clone() for _ in range(k)]
        geos = [(geo0[gk[0]].clone(), geo0[gk[1]].clone()) for _ in range(k)]
        res = torch.empty(k, dtype=torch.float64, device="cuda")

        def call_int(i):
            plan.set_geometry(dt, *geos[i])
            spx.integral(plan, ins[i], res[i])
        ms = timed_rotating(torch, call_int, k, 60, stream)
        plan.set_geometry(dt, geo0[gk[0]], geo0[gk[1]])
        ops[f"integral_{tag}"] = roof(ms, nbytes, E * op_flops_per_elem("integral", P, Q), False, hbm_peak, pk)
        ops[f"integral_{tag}"]["timing"] = f"{k} copies of the operands launched in turn from a CUDA graph"
        del ins, geos
    ex["ops_hex32"] = ops
    # variable order workload
    wv, pv, gv, cv = make_workload("hex3d_24_varp", spx, mesh, synth, torch)
    pv = pv[0]
    nb = sum(helm_bytes_per_elem(int(p_), int(p_) + 2, 1) for p_ in pv.orders)
    nfl = sum(helm_flops_per_elem(int(p_), int(p_) + 2) for p_ in pv.orders)
    var = {}
    for dt, sz in ((torch.float32, 4), (torch.float64, 8)):
        uu = torch.tensor(cv, device="cuda", dtype=dt)
        oo = torch.empty_like(uu)
        pv.autotune("helmholtz", dt, uu, oo, reps=5)
        ms = timed(lambda: spx.helmholtz(pv, uu, out=oo), reps, stream)
        tag = "f32" if dt == torch.float32 else "f64"
        r = roof(ms, nb * sz, nfl, dt == torch.float64, hbm_peak, fp64_peak if dt == torch.float64 else fp32_peak)
        r["gdofs"] = round(pv.n_coef / ms / 1e6, 3)
        r["tiles_eb_by_order"] = {int(p_): pv.get_tile("helmholtz", dt, int(p_))[0]
                                  for p_ in sorted(set(pv.orders.tolist()))}
        r["threads_stages"] = list(pv.get_tile("helmholtz", dt, int(pv.orders.min()))[1:])
        var[tag] = r
    var["flops_model"] = "sum over elements of the per-order Helmholtz flops (P_e, Q_e = P_e + 2)"
    ex["varp_hex24"] = var
    del pv, gv
    # GLL nodal basis (classical spectral elements) on the same 32^3 mesh, P = 4,
    # collocated on its Q = P + 1 = 5 GLL points: B = I, no B contractions
    try:
        ex["nodal_hex32_p4"] = measure_nodal(spx, mesh, synth, torch, stream, hbm_peak, fp64_peak, fp32_peak)
    except Exception as err:   # an extra: never lose the benchmark line over it
        ex["nodal_hex32_p4"] = {"error": str(err)[:200]}
    # collapsed-coordinate elements (prisms, triangles)
    try:
        ex["collapsed"] = measure_collapsed(spx, mesh, synth, torch, stream, hbm_peak, fp64_peak, fp32_peak)
    except Exception as err:   # an extra: never lose the benchmark line over it
        ex["collapsed"] = {"error": str(err)[:200]}
    # adjoint workload
    wa, pa, ga, ca = make_workload("hex3d_16_p6", spx, mesh, synth, torch)
    pa, ga = pa[0], ga[0]
    X = ga["xq"].reshape(pa.E, 3, 512)
    lam = (1.0 + 0.5 * torch.sin(torch.pi * X[:, 0])).reshape(-1).contiguous()
    kap = (1.0 + 0.3 * torch.cos(torch.pi * X[:, 1])).reshape(-1).contiguous()
    uu = torch.tensor(ca, device="cuda", requires_grad=True)
    ff = torch.tensor(synth.uniform(synth.rng(41), pa.n_coef), device="cuda")
    lp, kp = lam.clone().requires_grad_(True), kap.clone().requires_grad_(True)
    # the forward / backward Helmholtz and the adjoint kernel on autotuned tiles
    scratch = torch.empty(2 * pa.n_quad, dtype=torch.float64, device="cuda")
    pa.autotune("helmholtz", torch.float64, uu.detach(), torch.empty_like(ff), reps=2)
    pa.autotune("helmholtz_adjoint", torch.float64, uu.detach(), scratch, reps=2)

    def fwd_bwd():
        y = spx.helmholtz_ad(pa, uu, lp, kp)
        loss = 0.5 * ((y - ff) ** 2).sum()
        loss.backward()

    fwd_bwd()
    ms = timed(fwd_bwd, 10, stream)
    Pa, Qa = 6, 8
    na, qa = (Pa + 1) ** 3, Qa ** 3
    # forward H u and backward H g (each: coefficients in and out, 7 geometric
    # factors, lambda and kappa fields) + the adjoint kernel (u, g in; 7 factors;
    # g_lambda, g_kappa out); flops: three Helmholtz-sized passes (the adjoint's
    # two BwdTrans + gradients and its pointwise work equal one apply's count)
    nb_a = pa.E * 3 * (2 * na + 9 * qa) * 8
    nfl_a = pa.E * 3 * helm_flops_per_elem(Pa, Qa)
    r = roof(ms, nb_a, nfl_a, True, hbm_peak, fp64_peak)
    r["fwd_bwd_ms"] = r.pop("ms")
    r["model"] = "H u, H g and the adjoint kernel per step; torch's loss arithmetic not counted"
    ex["adjoint_hex16_p6"] = r
    del pa, ga
    # 2D correctness workload (16 x 16 affine quads, P = 4, Q = 6, FP64): BwdTrans,
    # IProduct and Helmholtz once each after warm-up; latency-sized (6400 DOFs),
    # so times only, no roofline
    try:
        ex["quad2d_16x16_p4"] = measure_quad2d(spx, mesh, synth, torch, stream)
    except Exception as err:   # an extra: never lose the benchmark line over it
        ex["quad2d_16x16_p4"] = {"error": str(err)[:200]}
    # periodic solve of the 48^3 workload
    ex["cg_hex48"] = measure_cg(spx, mesh, synth, torch, hbm_peak)
    return ex


def nodal_flops_per_elem(P):
    """Collocation Helmholtz (Q = P + 1): gradient and transposed gradient along
    three directions (6 Q^4 multiply-adds) + 20 flops per point."""
    Q = P + 1
    return 2 * 6 * Q ** 4 + 20 * Q ** 3


def measure_nodal(spx, mesh, synth, torch, stream, hbm_peak, fp64_peak, fp32_peak):
    w = synth.WORKLOADS["hex3d_32_p4"]
    N, P = w["N"], w["P"]
    Q = P + 1
    plan = spx.Plan(3, N ** 3, order=P, q_offset=1, basis={P: spx.nodal_basis_tables(P, Q)})
    g = spx.geom_factors(plan, mesh.structured_nodes(3, N, P, w["amp"]), want_xq=False)
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    coef = synth.uniform(synth.rng(w["seed"]), plan.n_coef)
    E = plan.E
    out = {"basis": "Lagrange through the P+1 GLL points, collocated (Q = P + 1): B = I", "P": P, "Q": Q}
    for dt, sz in ((torch.float64, 8), (torch.float32, 4)):
        u = torch.tensor(coef, device="cuda", dtype=dt)
        y = torch.empty_like(u)
        plan.autotune("helmholtz", dt, u, y, reps=3)
        ms = timed(lambda: spx.helmholtz(plan, u, out=y), 30, stream)
        fp64 = dt == torch.float64
        r = roof(ms, E * (2 * (P + 1) ** 3 + 7 * Q ** 3) * sz, E * nodal_flops_per_elem(P), fp64, hbm_peak,
                 fp64_peak if fp64 else fp32_peak)
        r["gdofs"] = round(plan.n_coef / ms / 1e6, 3)
        r["tile_eb_threads_stages"] = list(plan.get_tile("helmholtz", dt, P))
        out["f64" if fp64 else "f32"] = r
    del plan, g
    # the same basis on Q = P + 2 points: no parity of the modified basis, no
    # collocation, so the library's generic body (direct 1D contractions)
    Q2 = P + 2
    plan = spx.Plan(3, N ** 3, order=P, q_offset=2, basis={P: spx.nodal_basis_tables(P, Q2)})
    g = spx.geom_factors(plan, mesh.structured_nodes(3, N, P, w["amp"]), want_xq=False)
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    gen = {"Q": Q2, "body": "generic (any caller basis without the modified basis's parity)"}
    for dt, sz in ((torch.float64, 8), (torch.float32, 4)):
        u = torch.tensor(coef, device="cuda", dtype=dt)
        y = torch.empty_like(u)
        plan.autotune("helmholtz", dt, u, y, reps=3)
        ms = timed(lambda: spx.helmholtz(plan, u, out=y), 30, stream)
        fp64 = dt == torch.float64
        r = roof(ms, E * (2 * (P + 1) ** 3 + 7 * Q2 ** 3) * sz, E * helm_flops_per_elem(P, Q2), fp64, hbm_peak,
                 fp64_peak if fp64 else fp32_peak)
        r["gdofs"] = round(plan.n_coef / ms / 1e6, 3)
        r["tile_eb_threads_stages"] = list(plan.get_tile("helmholtz", dt, P))
        gen["f64" if fp64 else "f32"] = r
    out["q_plus_2_generic"] = gen
    return out


def collapsed_flops_per_elem(shape, P):
    """Algorithmic flops of the collapsed Helmholtz (Q = P + 2): BwdTrans and its
    transpose by the three (two) 1D stages, the ragged collapsed-direction one
    over n_T = (P+1)(P+2)/2 triangle modes, plus 6 Q^d+1 (4 Q^3 in 2D: 2 Q^2 Q)
    multiply-adds of the collocation gradient and its transpose and 20 flops per
    point."""
    n, Q = P + 1, P + 2
    nt = n * (n + 1) // 2
    if shape == "tri":
        bwd = nt * Q + n * Q * Q
        return 2 * (2 * bwd + 2 * 2 * Q ** 3) + 14 * Q ** 2
    if shape == "tet":
        ntet = n * (n + 1) * (n + 2) // 6
        bwd = ntet * Q + nt * Q * Q + n * Q ** 3
    else:
        bwd = n * nt * Q + n * n * Q * Q + n * Q ** 3
    return 2 * (2 * bwd + 6 * Q ** 4) + 20 * Q ** 3


def measure_collapsed(spx, mesh, synth, torch, stream, hbm_peak, fp64_peak, fp32_peak):
    """Helmholtz on the collapsed-element workloads (affine prisms / triangles of a skewed grid)."""
    out = {}
    for name in ("prism3d_24_p4", "tet3d_16_p4", "tri2d_128_p4"):
        w = synth.WORKLOADS[name]
        N, P, shape, d = w["N"], w["P"], w["shape"], w["dim"]
        plan = spx.Plan(d, (6 if shape == "tet" else 2) * N ** d, order=P, shape=shape)
        g = spx.geom_factors(plan, mesh.collapsed_vertices(shape, N), want_xq=False)
        plan.set_geometry(torch.float64, g["geom"], g["dxi"])
        plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
        coef = synth.uniform(synth.rng(w["seed"]), plan.n_coef)
        E, Q = plan.E, P + 2
        nm = plan.n_coef // E
        rec = {"elements": E, "modes_per_element": nm, "points_per_element": Q ** d}
        for dt, sz in ((torch.float64, 8), (torch.float32, 4)):
            u = torch.tensor(coef, device="cuda", dtype=dt)
            y = torch.empty_like(u)
            plan.autotune("helmholtz", dt, u, y, reps=3)
            fp64 = dt == torch.float64
            nbytes = E * (2 * nm + (7 if d == 3 else 4) * Q ** d) * sz
            # k copies of the operands and geometric factors (> 2 x L2), launched in turn from a CUDA graph
            k = max(2, -(-2 * L2_BYTES // nbytes))
            gk = ("geom", "dxi") if fp64 else ("geom32", "dxi32")
            us = [u.clone() for _ in range(k)]
            ys = [torch.empty_like(u) for _ in range(k)]
            geos = [(g[gk[0]].clone(), g[gk[1]].clone()) for _ in range(k)]

            def call(i, us=us, ys=ys, geos=geos, dt=dt):
                plan.set_geometry(dt, *geos[i])
                spx.helmholtz(plan, us[i], out=ys[i])
            ms = timed_rotating(torch, call, k, 60, stream)
            plan.set_geometry(dt, g[gk[0]], g[gk[1]])
            del us, ys, geos
            r = roof(ms, nbytes, E * collapsed_flops_per_elem(shape, P), fp64, hbm_peak,
                     fp64_peak if fp64 else fp32_peak)
            r["timing"] = f"{k} copies of the operands launched in turn from a CUDA graph"
            r["gdofs"] = round(plan.n_coef / ms / 1e6, 3)
            r["tile_eb_threads_stages"] = list(plan.get_tile("helmholtz", dt, P))
            rec["f64" if fp64 else "f32"] = r
        out[name] = rec
    return out


def measure_quad2d(spx, mesh, synth, torch, stream):
    w, plans, _, coef = make_workload("quad2d_16x16_p4", spx, mesh, synth, torch)
    plan = plans[0]
    u = torch.tensor(coef, device="cuda")
    f = spx.bwd_trans(plan, u)
    y, c = torch.empty_like(u), torch.empty_like(u)
    out = {}
    for op, fn in (("bwd_trans_us", lambda: spx.bwd_trans(plan, u, f)),
                   ("iproduct_us", lambda: spx.iproduct(plan, f, c)),
                   ("helmholtz_us", lambda: spx.helmholtz(plan, u, lam=1.0, out=y))):
        fn()
        out[op] = round(timed(fn, 50, stream) * 1e3, 2)
    out["elements"] = plan.E
    out["local_dofs"] = plan.n_coef
    return out


def measure_cg(spx, mesh, synth, torch, hbm_peak):
    import numpy as np
    w = synth.WORKLOADS["hex3d_48_p4"]
    N, P = w["N"], w["P"]
    plan = spx.Plan(3, N ** 3, order=P)
    g = spx.geom_factors(plan, mesh.structured_nodes(3, N, P, w["amp"]))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    l2g, ng = mesh.periodic_l2g(3, N, P)
    X = g["xq"].reshape(plan.E, 3, 216)
    u_star = torch.prod(torch.sin(2 * np.pi * X), dim=1).reshape(-1).contiguous()
    f = spx.assemble(plan, l2g, spx.iproduct(plan, (1.0 + 12 * np.pi ** 2) * u_star), ng)
    u32 = torch.empty(plan.n_coef, dtype=torch.float32, device="cuda")
    plan.autotune("helmholtz", torch.float32, u32.uniform_(), torch.empty_like(u32), reps=3)
    u64 = torch.rand(plan.n_coef, dtype=torch.float64, device="cuda")
    plan.autotune("helmholtz", torch.float64, u64, torch.empty_like(u64), reps=2)
    ws = torch.empty(max(spx.cg_workspace_bytes(plan, ng, p) for p in ("f64", "f32_refine")), dtype=torch.uint8,
                     device="cuda")
    res = {"global_dofs": ng, "local_dofs": plan.n_coef, "tol": 1e-10,
           "timing": "wall clock of the whole cg_solve call (CSR build, Jacobi diagonal, FP64 residuals, "
                     "graph capture, iterations), synchronised on both sides"}
    # f32_refine: FP32 PCG restarted after each FP64 refinement step (inner_tol 1e-5);
    # f32_reliable: one FP32 PCG run whose residual is replaced by the FP64 one every 1e-2 reduction
    for prec, itol in (("f32_reliable", 1e-2), ("f32_refine", 1e-5), ("f64", 1e-5)):
        spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-10, precision=prec, workspace=ws, maxit=5,
                     raise_on_fail=False)  # warm-up (graphs, tiles)
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            t0 = time.perf_counter()
            x, info = spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-10, precision=prec, inner_tol=itol, workspace=ws)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        uh = spx.bwd_trans(plan, spx.gather(plan, l2g, x))
        res[prec] = {"time_s": round(t, 4), "iters": info["iters"], "outer_iters": info["outer_iters"],
                     "clocks": clk.summary(),
                     "inner_tol": itol if prec != "f64" else None,
                     "rel_residual": info["rel_residual"], "status": info["status"],
                     "max_err_vs_exact": (uh - u_star).abs().max().item()}
    # one FP32 iteration: time from two iteration caps of one FP32 run, and the
    # algorithmic bytes it moves (Helmholtz apply + gather + assembly + vector updates)
    ts = {}
    for m in (50, 250):
        spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-14, precision="f32_reliable", maxit=5, max_outer=1, workspace=ws,
                     raise_on_fail=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf = spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-14, precision="f32_reliable", maxit=m, max_outer=1,
                              workspace=ws, raise_on_fail=False)
        torch.cuda.synchronize()
        ts[m] = (time.perf_counter() - t0, inf["iters"])
    per = (ts[250][0] - ts[50][0]) / max(1, ts[250][1] - ts[50][1])
    nl, E = plan.n_coef, plan.E
    it_bytes = (E * helm_bytes_per_elem(P, P + 2, 4)            # Helmholtz apply
                + nl * 4 * 2 + ng * 4                           # gather: l2g, local copy, p
                + (ng + 1) * 4 + nl * 4 * 2 + ng * 4 * 2        # assembly: row_ptr, cols, ql, p, q
                + ng * 4 * 8 + ng * 4 * 3)                      # update (5 reads, 3 writes), direction
    res["f32_iteration"] = {"us": round(per * 1e6, 1), "algorithmic_bytes": it_bytes,
                            "gbs": round(it_bytes / per / 1e9, 1), "hbm_frac": round(it_bytes / per / 1e9 / hbm_peak, 4),
                            "timing": "difference of 250- and 50-iteration FP32 runs (wall clock, synchronised)"}
    res["speedup_f32_refine_vs_f64"] = round(res["f64"]["time_s"] / res["f32_refine"]["time_s"], 3)
    res["speedup_f32_reliable_vs_f64"] = round(res["f64"]["time_s"] / res["f32_reliable"]["time_s"], 3)
    return res


def run_case(a):
    """Single-purpose runs for profiling (ncu launch lists and captures): one
    workload, one operation, a short JSON line; not the benchmark contract."""
    import torch
    import paper_1906_03489_gb300 as spx
    from paper_1906_03489_gb300 import mesh, synth
    dist_setup()
    spx.lib()
    stream = torch.cuda.current_stream()
    if a.case == "cg":
        w = synth.WORKLOADS["hex3d_48_p4"]
        N, P = w["N"], w["P"]
        plan = spx.Plan(3, N ** 3, order=P)
        g = spx.geom_factors(plan, mesh.structured_nodes(3, N, P, w["amp"]))
        plan.set_geometry(torch.float64, g["geom"], g["dxi"])
        plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
        l2g, ng = mesh.periodic_l2g(3, N, P)
        f = torch.tensor(synth.uniform(synth.rng(w["seed"]), ng), device="cuda")
        spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-10, precision=a.precision, maxit=5, max_outer=1,
                     raise_on_fail=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-10, precision=a.precision, maxit=a.cg_maxit,
                               max_outer=1, raise_on_fail=False)
        torch.cuda.synchronize()
        print(json.dumps({"case": "cg", "workload": "hex3d_48_p4", "precision": a.precision,
                          "iters": info["iters"], "s": round(time.perf_counter() - t0, 4)}), flush=True)
    elif a.case == "helm":
        w, plans, _, coef = make_workload(a.workload, spx, mesh, synth, torch)
        plan = plans[0]
        P = w["P"]
        dt = torch.float64 if a.precision == "f64" else torch.float32
        u = torch.tensor(coef, device="cuda", dtype=dt)
        y = torch.empty_like(u)
        tile = a.tile64 if dt == torch.float64 else a.tile
        if tile:   # a reproducible launch without autotuning
            eb, nt, st = (int(x) for x in tile.split(","))
            plan.set_tile("helmholtz", dt, eb, nt, st)
        else:
            plan.autotune("helmholtz", dt, u, y, reps=2)
        spx.helmholtz(plan, u, out=y)   # warm-up (module load, tile lists)
        ms = timed(lambda: spx.helmholtz(plan, u, out=y), max(1, a.steps), stream)
        print(json.dumps({"case": "helm", "workload": a.workload, "dtype": str(dt), "ms": round(ms, 4),
                          "tile": plan.get_tile("helmholtz", dt, P)}), flush=True)
    elif a.case == "ops":
        # BwdTrans then IProductWRTBase of the workload, each with the same fixed tile (--tile / --tile64)
        w, plans, _, coef = make_workload(a.workload, spx, mesh, synth, torch)
        plan = plans[0]
        P = w["P"]
        dt = torch.float64 if a.precision == "f64" else torch.float32
        c = torch.tensor(coef, device="cuda", dtype=dt)
        f = torch.empty(plan.n_quad, dtype=dt, device="cuda")
        tile = a.tile64 if dt == torch.float64 else a.tile
        res = {"case": "ops", "workload": a.workload, "dtype": str(dt)}
        for op, fn in (("bwd_trans", lambda: spx.bwd_trans(plan, c, f)), ("iproduct", lambda: spx.iproduct(plan, f, c))):
            t_op = a.tile_iprod if (op == "iproduct" and a.tile_iprod) else tile
            if t_op:
                eb, nt, st = (int(x) for x in t_op.split(","))
                plan.set_tile(op, dt, eb, nt, st)
            fn()   # warm-up (module load, tile lists)
            res[op + "_ms"] = round(timed(fn, max(1, a.steps), stream), 4)
            res[op + "_tile"] = plan.get_tile(op, dt, P)
        print(json.dumps(res), flush=True)
    elif a.case == "collapsed":
        # Helmholtz on a collapsed-element workload (--workload prism3d_24_p4 | tet3d_16_p4 | tri2d_128_p4)
        w = synth.WORKLOADS[a.workload]
        N, P, shape, d = w["N"], w["P"], w["shape"], w["dim"]
        plan = spx.Plan(d, (6 if shape == "tet" else 2) * N ** d, order=P, shape=shape)
        g = spx.geom_factors(plan, mesh.collapsed_vertices(shape, N), want_xq=False)
        plan.set_geometry(torch.float64, g["geom"], g["dxi"])
        plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
        dt = torch.float64 if a.precision == "f64" else torch.float32
        u = torch.tensor(synth.uniform(synth.rng(w["seed"]), plan.n_coef), device="cuda", dtype=dt)
        y = torch.empty_like(u)
        tile = a.tile64 if dt == torch.float64 else a.tile
        if tile:
            eb, nt, st = (int(x) for x in tile.split(","))
            plan.set_tile("helmholtz", dt, eb, nt, st)
        else:
            plan.autotune("helmholtz", dt, u, y, reps=3)
        spx.helmholtz(plan, u, out=y)   # warm-up
        ms = timed(lambda: spx.helmholtz(plan, u, out=y), max(1, a.steps), stream)
        print(json.dumps({"case": "collapsed", "workload": a.workload, "dtype": str(dt), "ms": round(ms, 4),
                          "tile": plan.get_tile("helmholtz", dt, P)}), flush=True)
    elif a.case == "peaks":
        print(json.dumps({"case": "peaks", "fp_peaks": fp_peaks(torch)}), flush=True)
    elif a.case == "varp":
        w, plans, _, coef = make_workload("hex3d_24_varp", spx, mesh, synth, torch)
        plan = plans[0]
        dt = torch.float32 if a.precision != "f64" else torch.float64
        u = torch.tensor(coef, device="cuda", dtype=dt)
        y = torch.empty_like(u)
        if a.varp_tiles:   # elements per tile of orders 2..8 (no autotuning: a reproducible launch)
            # optional 8th and 9th fields: threads class (FP32: the highest paired order) and stages
            f = [int(x) for x in a.varp_tiles.split(",")]
            nt = f[7] if len(f) > 7 else 512
            st = f[8] if len(f) > 8 else (0 if dt == torch.float32 else 2)
            for P, eb in zip(range(2, 9), f[:7]):
                plan.set_tile("helmholtz", dt, eb, nt, st, order=P)
        else:
            plan.autotune("helmholtz", dt, u, y, reps=5)
        spx.helmholtz(plan, u, out=y)   # warm-up (module load, tile lists)
        ms = timed(lambda: spx.helmholtz(plan, u, out=y), max(1, a.steps), stream)
        orders = sorted(set(plan.orders.tolist()))
        print(json.dumps({"case": "varp", "workload": "hex3d_24_varp", "dtype": str(dt), "ms": round(ms, 4),
                          "tiles": {int(P): plan.get_tile("helmholtz", dt, int(P))[0] for P in orders},
                          "threads_stages": plan.get_tile("helmholtz", dt, int(orders[0]))[1:]}), flush=True)


def oracle_sample_rate(name, n_elem_sample, seconds, repeat=None):
    """Times the oracle's dense Helmholtz on a sample of the workload's elements."""
    import numpy as np
    from oracle import operators
    from oracle.geometry import StructuredMesh
    from paper_1906_03489_gb300 import synth
    w = synth.WORKLOADS[name]
    P, Q = w["P"], w["P"] + 2
    # a sub-mesh of the same elements (same order, quadrature and curvature)
    n_side = max(1, round(n_elem_sample ** (1.0 / 3.0)))
    m = StructuredMesh(3, n_side, P, amp=w["amp"])
    m.geometry(P, Q, np.arange(m.E))          # geometry precomputed, as on the GPU
    u = synth.uniform(synth.rng(w["seed"]), m.coef_off[-1])
    operators.helmholtz(m, u)                  # warm-up
    t0 = time.perf_counter()
    reps = 0
    while True:
        operators.helmholtz(m, u)
        reps += 1
        el = time.perf_counter() - t0
        if (repeat is not None and reps >= repeat) or (repeat is None and el >= seconds):
            break
    return m.E * (P + 1) ** 3 * reps / el / 1e9, m.E, reps, el


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the architecture)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(name, seconds=15.0):
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rate, ne, reps, el = oracle_sample_rate(name, 4096, seconds)
    return {"value": round(rate, 6), "unit": "GDOF/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "host_cpus": os.cpu_count(),
            "sample": f"dense FP64 oracle Helmholtz on a {ne}-element sub-mesh of the same curved P=4 hexes, "
                      f"{reps} applies in {el:.1f} s (numpy/OpenBLAS, {cores} threads)"}


def run_reference(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    name = a.workload
    # warm-up steps, then K timed steps; each step = one dense apply on the sample
    rate, ne, reps, el = oracle_sample_rate(name, 512, None, repeat=max(1, a.steps))
    ms = el / max(1, reps) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": round(rate, 6), "unit": "GDOF/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample_elements": ne},
            "cpu_baseline": {"value": round(rate, 6), "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "host_cpus": os.cpu_count(),
                             "sample": f"dense FP64 oracle Helmholtz, {ne}-element sub-mesh of the same "
                                       f"curved hexes per step"},
            "e2e": {"value": round(rate, 6), "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hex3d_32_p4")
    ap.add_argument("--tile", default=None, help="FP32 apply: eb,threads,stages (skips autotuning)")
    ap.add_argument("--tile64", default=None, help="FP64 apply: eb,threads,stages (skips autotuning)")
    ap.add_argument("--tile-iprod", dest="tile_iprod", default=None,
                    help="--case ops: IProductWRTBase tile when it differs from BwdTrans's")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--case", default="bench", choices=["bench", "cg", "varp", "helm", "ops", "collapsed", "peaks"],
                    help="bench: the benchmark line; cg / varp / helm / ops / collapsed / peaks: one short run "
                         "for profiling")
    ap.add_argument("--precision", default="f32_reliable",
                    help="cg: f64 | f32_refine | f32_reliable; varp, helm: f32 | f64")
    ap.add_argument("--cg-maxit", type=int, default=30)
    ap.add_argument("--varp-tiles", default=None, help="varp: elements per tile of orders 2..8, e.g. 24,16,8,4,3,2,2")
    a = ap.parse_args()
    a.warmup = max(3, a.warmup)
    if a.case != "bench":
        run_case(a)
    elif a.impl == "reference":
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        os.environ.setdefault("OPENBLAS_NUM_THREADS", os.environ["OMP_NUM_THREADS"])
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
