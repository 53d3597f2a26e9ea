#!/usr/bin/env python
"""Benchmark of the spectral/hp Helmholtz operator on GB300.

A step is one application of the Helmholtz operator H = lambda M + L (BwdTrans,
reference gradient, pointwise geometric factors, transposed gradient and
IProductWRTBase fused in one kernel launch) to every element of the workload
mesh: by default 32^3 curved hexes, P = 4, Q = 6, the operator applied in FP32
(the precision whose roofline is HBM).  Prints one JSON line.

Besides the timed steps it reports, each measured separately after the timed
region: the FP64 apply of the same workload (ALU roofline), PhysDeriv, the
variable-order workload (24^3 hexes, P_e in 2..8), the adjoint workload (16^3
hexes, P = 6) and the periodic solve of the 48^3 workload to a 1e-10 relative
residual in FP32-inner + FP64 refinement (restarted, and with reliable updates)
and in all-FP64 CG.

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


# FP64 ALU peak: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def helm_bytes_per_elem(P, Q, sz, dim=3):
    n = P + 1
    return (2 * n ** dim + (7 if dim == 3 else 4) * Q ** dim) * sz


def helm_flops_per_elem(P, Q):
    n = P + 1
    bwd = n ** 3 * Q + n ** 2 * Q ** 2 + n * Q ** 3
    return 2 * (2 * bwd + 6 * Q ** 4) + 20 * Q ** 3


# Sources of the FP32 Helmholtz kernel and its launcher (what its ncu counters depend on).
HELM_SOURCES = ("helm_pair.cuh", "op_kernel.cuh", "lanes.cuh", "kernel_params.h", "device_common.cuh",
                "launch_ops.cuh", "smem_layout.h")


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


def profiled_traffic(name):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_digest") == kernel_digest(HELM_SOURCES):
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
    dt = torch.float32
    u = [torch.tensor(coef, device="cuda", dtype=dt) for _ in plans]
    out = [torch.empty_like(x) for x in u]
    if a.tile:
        eb, nt, st = (int(x) for x in a.tile.split(","))
        for p in plans:
            p.set_tile("helmholtz", dt, eb, nt, st)
    else:
        plans[0].autotune("helmholtz", dt, u[0], out[0], reps=5)
        tile = plans[0].get_tile("helmholtz", dt, P)
        plans[1].set_tile("helmholtz", dt, *tile)
    tile = plans[0].get_tile("helmholtz", dt, P)

    def step(i):
        k = i & 1
        spx.helmholtz(plans[k], u[k], lam=1.0, out=out[k])

    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(a.steps):
            step(i)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    barrier(world)
    ms = max_over_ranks(ms, world)
    dofs = E * (P + 1) ** 3
    value = world * dofs / (ms * 1e-3) / 1e9
    bytes_launch = E * helm_bytes_per_elem(P, Q, 4)
    achieved = bytes_launch / (ms * 1e-3) / 1e9
    traffic = profiled_traffic("helmholtz_f32_hex32.txt")

    # end to end through the C ABI with host buffers: every step copies its
    # input u from pinned host memory, applies the operator and copies the
    # result y back.  Served as a pipeline on three streams with two device
    # buffers each: the upload of step i+1 and the download of step i-1 run on
    # the copy engines while step i computes.
    uh = torch.tensor(coef, dtype=dt).pin_memory()
    yh = [torch.empty(plans[0].n_coef, dtype=dt).pin_memory() for _ in range(2)]
    ud = [torch.empty_like(u[0]) for _ in range(2)]
    yd = [torch.empty_like(u[0]) for _ in range(2)]
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
            spx.helmholtz(plans[0], ud[k], lam=1.0, out=yd[k])
            ev_comp[k].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[k])
            yh[k].copy_(yd[k], non_blocking=True)
            ev_out[k].record(s_out)

    for i in range(4):
        e2e_step(i)
    torch.cuda.synchronize()
    k_e2e = max(10, a.steps // 10)
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(s_in)
    for i in range(k_e2e):
        e2e_step(i)
    t1e.record(s_out)          # after the last download, which follows every earlier step
    t1e.synchronize()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(t0e.elapsed_time(t1e) / k_e2e, world)
    e2e_value = world * dofs / (ms_e2e * 1e-3) / 1e9

    extras = {}
    if a.extras and rank == 0:
        extras = measure_extras(spx, mesh, synth, torch, plans, geoms, coef, stream, hbm_peak)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(name, seconds=a.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GDOF/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name, "mesh": f"{w['N']}^3 curved hexes (x'=x+{w['amp']} sin2piy sin2piz)",
                       "P": P, "Q": Q, "elements_per_gpu": E, "local_dofs_per_gpu": dofs,
                       "op": "Helmholtz H=lambda M+L, lambda=1, unassembled, FP32 FMA/FP32 accumulate",
                       "tile_eb_threads_stages": list(tile),
                       "l2": f"inputs {2 * bytes_launch / 1e6:.0f} MB per step pair alternate between two "
                             f"independent copies (> {L2_BYTES / 1e6:.0f} MB L2): no L2 flush",
                       "parallelism": f"replica per GPU x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
                         "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": bytes_launch,
                         "bytes_model": "per element (2 (P+1)^3 coefficients + 7 Q^3 geometric factors) x 4 B"},
            "e2e": {"value": round(e2e_value, 3), "unit": "GDOF/s", "h2d_bytes_per_step": int(uh.numel() * 4),
                    "d2h_bytes_per_step": int(yh[0].numel() * 4), "ms_per_step": round(ms_e2e, 4),
                    "steps": k_e2e,
                    "pipeline": "pinned host buffers; 3 streams, 2 device buffers each: the upload of step i+1 "
                                "and the download of step i-1 overlap the apply of step i"},
            "gpu_launches": a.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_extras(spx, mesh, synth, torch, plans, geoms, coef, stream, hbm_peak):
    """Other operators / precisions / workloads, each timed after warm-up with CUDA events."""
    ex = {}
    plan = plans[0]
    P, Q, E = 4, 6, plan.E
    reps = 30
    # FP64 Helmholtz: ALU bound
    u64 = torch.tensor(coef, device="cuda")
    o64 = torch.empty_like(u64)
    plan.autotune("helmholtz", torch.float64, u64, o64, reps=3)
    ms = timed(lambda: spx.helmholtz(plan, u64, out=o64), reps, stream)
    fl = E * helm_flops_per_elem(P, Q)
    ex["fp64"] = {"helmholtz_gdofs": round(E * 125 / ms / 1e6, 3), "ms": round(ms, 4),
                  "roofline": {"bound": "alu", "achieved": round(fl / ms / 1e9, 4),
                               "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                               "frac": round(fl / ms / 1e9 / FP64_PEAK_TFLOPS, 4),
                               "flops_per_launch": fl},
                  "hbm_frac": round(E * helm_bytes_per_elem(P, Q, 8) / ms / 1e6 / hbm_peak, 4)}
    # PhysDeriv, BwdTrans, IProduct (FP32 and FP64), each with its autotuned tile
    ops = {}
    for dt, sz in ((torch.float32, 4), (torch.float64, 8)):
        c = torch.tensor(coef, device="cuda", dtype=dt)
        f = spx.bwd_trans(plan, c)
        outs = [torch.empty_like(f) for _ in range(3)]
        tag = "f32" if dt == torch.float32 else "f64"
        packed = torch.empty(3 * plan.n_quad, dtype=dt, device="cuda")
        for op, fn, nbytes, tin, tout in (
                ("phys_deriv", lambda: spx.phys_deriv(plan, f, outs), E * 13 * Q ** 3 * sz, f, packed),
                ("bwd_trans", lambda: spx.bwd_trans(plan, c, f), E * (125 + Q ** 3) * sz, c, f),
                ("iproduct", lambda: spx.iproduct(plan, f, c), E * (2 * Q ** 3 + 125) * sz, f, c)):
            plan.autotune(op, dt, tin, tout, reps=5)
            fn()
            ms = timed(fn, reps, stream)
            ops[f"{op}_{tag}"] = {"ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
                                  "hbm_frac": round(nbytes / ms / 1e6 / hbm_peak, 4),
                                  "tile_eb_threads_stages": list(plan.get_tile(op, dt, P))}
        # FwdTrans (elemental preconditioned CG in one launch; reads f and JW, writes the coefficients)
        # and Integral (reads f and JW)
        f = spx.bwd_trans(plan, torch.tensor(coef, device="cuda", dtype=dt))
        cf = torch.empty(plan.n_coef, dtype=dt, device="cuda")
        plan.autotune("fwd_trans", dt, f, cf, reps=3)
        ms = timed(lambda: spx.fwd_trans(plan, f, cf), reps, stream)
        nbytes = E * (2 * Q ** 3 + 125) * sz
        ops[f"fwd_trans_{tag}"] = {"ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
                                   "hbm_frac": round(nbytes / ms / 1e6 / hbm_peak, 4),
                                   "tile_eb_threads_stages": list(plan.get_tile("fwd_trans", dt, P)),
                                   "max_err_vs_input_coefficients": (cf.double() - torch.tensor(coef, device="cuda")
                                                                     ).abs().max().item()}
        if dt == torch.float64:   # adaptive-order sensor (FP64): reads the coefficients and JW, writes one value per element
            cc = torch.tensor(coef, device="cuda")
            so = torch.empty(plan.E, dtype=torch.float64, device="cuda")
            plan.autotune("sensor", dt, cc, so, reps=3)
            ms = timed(lambda: spx.sensor(plan, cc, so), reps, stream)
            nbytes = E * (125 + Q ** 3 + 1) * sz
            ops["sensor_f64"] = {"ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
                                 "hbm_frac": round(nbytes / ms / 1e6 / hbm_peak, 4),
                                 "tile_eb_threads_stages": list(plan.get_tile("sensor", dt, P))}
        res = torch.empty((), dtype=torch.float64, device="cuda")
        ms = timed(lambda: spx.integral(plan, f, res), reps, stream)
        nbytes = E * 2 * Q ** 3 * sz
        ops[f"integral_{tag}"] = {"ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
                                  "hbm_frac": round(nbytes / ms / 1e6 / hbm_peak, 4)}
    ex["ops_hex32"] = ops
    # variable order workload
    wv, pv, gv, cv = make_workload("hex3d_24_varp", spx, mesh, synth, torch)
    pv = pv[0]
    nb = sum(helm_bytes_per_elem(int(p_), int(p_) + 2, 1) for p_ in pv.orders)
    var = {}
    for dt, sz in ((torch.float32, 4), (torch.float64, 8)):
        uu = torch.tensor(cv, device="cuda", dtype=dt)
        oo = torch.empty_like(uu)
        pv.autotune("helmholtz", dt, uu, oo, reps=2)
        ms = timed(lambda: spx.helmholtz(pv, uu, out=oo), reps, stream)
        tag = "f32" if dt == torch.float32 else "f64"
        var[tag] = {"ms": round(ms, 4), "gdofs": round(pv.n_coef / ms / 1e6, 3),
                    "gbs": round(nb * sz / ms / 1e6, 1), "hbm_frac": round(nb * sz / ms / 1e6 / hbm_peak, 4),
                    "tiles_eb_by_order": {int(p_): pv.get_tile("helmholtz", dt, int(p_))[0]
                                          for p_ in sorted(set(pv.orders.tolist()))}}
    ex["varp_hex24"] = var
    del pv, gv
    # adjoint workload
    wa, pa, ga, ca = make_workload("hex3d_16_p6", spx, mesh, synth, torch)
    pa, ga = pa[0], ga[0]
    X = ga["xq"].reshape(pa.E, 3, 512)
    lam = (1.0 + 0.5 * torch.sin(torch.pi * X[:, 0])).reshape(-1).contiguous()
    kap = (1.0 + 0.3 * torch.cos(torch.pi * X[:, 1])).reshape(-1).contiguous()
    uu = torch.tensor(ca, device="cuda", requires_grad=True)
    ff = torch.tensor(synth.uniform(synth.rng(41), pa.n_coef), device="cuda")
    lp, kp = lam.clone().requires_grad_(True), kap.clone().requires_grad_(True)

    def fwd_bwd():
        y = spx.helmholtz_ad(pa, uu, lp, kp)
        loss = 0.5 * ((y - ff) ** 2).sum()
        loss.backward()

    fwd_bwd()
    ms = timed(fwd_bwd, 10, stream)
    ex["adjoint_hex16_p6"] = {"fwd_bwd_ms": round(ms, 3)}
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
    elif a.case == "varp":
        w, plans, _, coef = make_workload("hex3d_24_varp", spx, mesh, synth, torch)
        plan = plans[0]
        dt = torch.float32 if a.precision != "f64" else torch.float64
        u = torch.tensor(coef, device="cuda", dtype=dt)
        y = torch.empty_like(u)
        if a.varp_tiles:   # elements per tile of orders 2..8 (no autotuning: a reproducible launch)
            for P, eb in zip(range(2, 9), (int(x) for x in a.varp_tiles.split(","))):
                plan.set_tile("helmholtz", dt, eb, 512, 0 if dt == torch.float32 else 2, order=P)
        else:
            plan.autotune("helmholtz", dt, u, y, reps=2)
        spx.helmholtz(plan, u, out=y)   # warm-up (module load, tile lists)
        ms = timed(lambda: spx.helmholtz(plan, u, out=y), max(1, a.steps), stream)
        print(json.dumps({"case": "varp", "workload": "hex3d_24_varp", "dtype": str(dt), "ms": round(ms, 4),
                          "tiles": {int(P): plan.get_tile("helmholtz", dt, int(P))[0]
                                    for P in sorted(set(plan.orders.tolist()))}}), flush=True)


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


def cpu_baseline(name, seconds=15.0):
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rate, ne, reps, el = oracle_sample_rate(name, 4096, seconds)
    return {"value": round(rate, 6), "unit": "GDOF/s", "cores": cores, "kind": "oracle",
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
                             "sample": f"dense FP64 oracle Helmholtz, {ne}-element sub-mesh of the same "
                                       f"curved hexes per step"},
            "e2e": {"value": round(rate, 6), "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hex3d_32_p4")
    ap.add_argument("--tile", default=None, help="eb,threads,stages (skips autotuning)")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--case", default="bench", choices=["bench", "cg", "varp"],
                    help="bench: the benchmark line; cg / varp: one short run for profiling")
    ap.add_argument("--precision", default="f32_reliable", help="cg: f64 | f32_refine | f32_reliable; varp: f32 | f64")
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
