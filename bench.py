"""Throughput of hierarchical probing on the 32^3x64 Wilson-Dirac workload.

One step = one pass of the whole path over one block of probing vectors:
probe generation on the device, full spin-colour dilution (12 sources per
probe), mixed-precision BiCGStab with FP64 reliable updates to a true
relative residual 1e-10, the FP64 quadratures q_m = sum_a v^H x and the
incremental prefix T_s (the next block resumes the nested sequence where the
previous one stopped).  Metric: probing solves/s (one solve = one diluted
right-hand side converged), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: ranks take disjoint probe blocks (weak scaling, no collective on
the data path); the timing is the max over ranks.  ``--impl reference`` times
the CPU oracle (plain numpy BiCGStab) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 64)
KAPPA, EPS, LINK_SEED, Z0_SEED, TOL = 0.12, 0.4, 1003, 2003, 1e-10
METRIC = "probing solves/s (32^3x64 Wilson, mixed precision, true residual 1e-10)"
UNIT = "solves/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK = 6800.0
FP64_TFLOPS = 1.25   # nominal dense FP64 rate of a GB300
# mean iterations per solve of this workload with the oracle's algorithm (unpreconditioned BiCGStab
# in FP64), measured with the library's FP64 solver on a GB300 (12 right-hand sides, 44.75)
FP64_ITERS_PER_SOLVE = 44.75


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def source_hash(kernel):
    """Hash of the sources a kernel is built from: the shared field and geometry headers, the
    two-right-hand-side even-odd kernels, and the kernel's own definition in the solver templates
    (its DRAM traffic below is valid for them only)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1302_4018_gb300", "csrc")
    for f in ("hp_fields.cuh", "hp_internal.h", "hp_eo2.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "hp_wilson_impl.cuh")) as fh:
        text = fh.read()
    for name in (kernel, "eo_hop", "eo_site", "site_diag", "add_diag"):   # the kernel and its helpers
        i = text.find(" %s(" % name)
        if i >= 0:
            h.update(text[text.rfind("\n\n", 0, i):text.find("\n}\n", i)].encode())
    return h.hexdigest()[:12]


# DRAM traffic of the dominant kernel per byte of algorithmic work, from one ncu capture of the
# same kernel (k_eo2_even, the two-right-hand-side even-site stencil, eo_kernel 4) on 32^3x16 with
# 12 slots: 282.3 MB read + 143.3 MB written per launch against 377.5 MB algorithmic (12-real links;
# both parts of the launch -- spinors and links -- grow with the units processed, so the ratio
# carries over to the 32^3x64 launch); valid only for the kernel source it was taken on
NCU_TRAFFIC = {("k_eo_even", "f7f32fc9b7f5"): {"bytes_all_slots": 282.3e6 + 143.3e6,
                                      "alg_bytes_all_slots": 262144 * 104 * 12 + 4 * 524288 * 24}}


class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl"
        try:
            import torch

            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, value, device):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ algorithmic bytes
def spinor_link_bytes(prec):
    """(spinor bytes per site, algorithmic link bytes per link, bytes per site of the solution
    increment e): fp16/bf16 spinors carry a 4-byte norm per site, e is kept in the iteration
    precision; the link bytes are the per-unit figures of the Wilson roofline (FP64 18 reals,
    FP32 and FP16 / BF16 12 reals), although the mixed-precision stencils read the 18-real form
    (72 / 36 bytes) -- the extra bytes show in the measured DRAM traffic, not in the algorithmic
    count."""
    return {"fp64": (192, 144, 192), "fp32": (96, 48, 96), "fp16": (52, 24, 52), "bf16": (52, 24, 52)}[prec]


def kernel_bytes(name, prec, V, c):
    """Algorithmic DRAM bytes of one solver kernel over the run: every vector it touches read or
    written once, the links once per launch.  c: counts of the run -- rhs_iters (right-hand-side
    iterations), launches (of this kernel), exact (true-residual evaluations, including the
    initial one), groups (FP32 group updates), eo (iterating on the odd half)."""
    S, L, E = spinor_link_bytes(prec)
    X = 192                                   # FP64 or float-float solution, per site
    n, it, la = c["eo"], c["rhs_iters"], c["launches"]
    Vf = V // 2 if n else V                   # sites of the iterated vectors
    links = 4 * V * L * la
    if c.get("clover") and (name.startswith("k_eo_even") or name.startswith("k_eo_odd") or name.startswith("k_bicg_v")
                            or name.startswith("k_bicg_t")):
        links += Vf * 288 * la                # the FP32 clover blocks of the sites written, once per launch
    if name.startswith("k_bicg_v"):
        return Vf * 3 * S * it + links
    if name.startswith("k_bicg_t"):
        return Vf * 2 * S * it + links
    if name == "k_bicg_s":
        return Vf * 3 * S * it
    if name == "k_bicg_xr":
        return Vf * (5 * S + 2 * E) * it
    if name == "k_bicg_p":
        return Vf * 4 * S * it
    if name == "k_ru_accum":                  # x += e after group and exact updates (upper bound)
        return Vf * (2 * X + 2 * E) * (c["groups"] + c["updates"])
    if name.startswith("k_ru_residual"):
        return V * (X + 2 * S) * c["exact"] + 4 * V * 144 * la
    if name == "k_eo_even":                   # V and T steps: mid = d_e^-1 H_eo in
        return Vf * 2 * S * 2 * it + links
    if name.startswith("k_eo_odd_v"):         # v = d_o p - k^2 H_oe mid, (r^, v)
        return Vf * 4 * S * it + links
    if name.startswith("k_eo_odd_t"):         # t = d_o s - k^2 H_oe mid, (t, s), (t, t)
        return Vf * 3 * S * it + links
    if name == "k_eo_even<grp>":              # mid32 = d_e^-1 H_eo e (FP32)
        return Vf * (E + 96) * c["groups"] + 4 * V * 48 * la
    if name == "k_eo_odd<grp>":               # r_g -= d_o e - k^2 H_oe mid32; r = r_g; dots
        return Vf * (96 + E + 2 * 96 + 2 * S) * c["groups"] + 4 * V * 48 * la
    if name.startswith("k_eo_x1"):            # x_e = d_e^-1 (b_e + k H_eo x_o)
        return Vf * 2 * X * c["exact"] + 4 * V * 144 * la
    if name.startswith("k_eo_x2"):            # r_o = b_o - d_o x_o + k H_oe x_e
        return Vf * (2 * X + 2 * S + 96) * c["exact"] + 4 * V * 144 * la
    return None


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    from paper_1302_4018_gb300 import hprobe, synth

    ws, rank, local = dist_setup()
    device = "cuda:%d" % local
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(local, stream=stream.cuda_stream)
    U = synth.gauge_links(DIMS, EPS, LINK_SEED, device=device)
    V = U.shape[0]
    links_dev = torch.from_numpy(U.view(np.float64).reshape(-1)).to(device)
    links_host = torch.from_numpy(U.view(np.float64).reshape(-1)).pin_memory()
    del U
    from paper_1302_4018_gb300.sharding import gather_quadratures, probe_block

    prec = args.precision
    P = args.probes_per_step
    rounds = args.warmup + args.steps + 4
    q = np.zeros((rounds * ws + 1) * P + args.fp64_probes + 16, dtype=np.complex128)
    round_no = [0]

    def next_first():
        # rank r solves block r of every round (disjoint probes: the other ranks' entries of q stay 0
        # here until the all-gather at the end of the timed steps)
        first, _ = probe_block(rank, ws, P, round_no[0])
        round_no[0] += 1
        return first

    def step(first, links, precision=prec, probes=P, rhs_block=args.rhs_block):
        op = ctx.make_operator(hprobe.OP_WILSON, 0.0, KAPPA, links, None, csw=args.csw)
        s_max = first + probes
        opts = ctx.make_opts(precision, z0_seed=Z0_SEED, first=first, rhs_block=rhs_block,
                             even_odd=1 if args.even_odd else 0, eo_kernel=args.eo_kernel,
                             rhs_per_thread=args.rhs_per_thread, use_graph=args.use_graph)
        qq = q[:s_max].copy()
        T, qq, st = ctx.trace_inv(op, DIMS, s_max, TOL, opts, q_inout=qq)
        q[:s_max] = qq
        return st

    for _ in range(args.warmup):
        step(next_first(), links_dev)
    ctx.profile_enable(True)
    ctx.profile_report()
    clocks = Clocks(local)
    n0 = ctx.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step(next_first(), links_dev))
    # the nested estimate over every probe solved so far: at N > 1 one all-gather of the ranks' FP64
    # quadratures, then the prefix sums by the library's kernel (a one-rank run's T_s, bit for bit)
    s_done = round_no[0] * ws * P
    q_all = gather_quadratures(q, rank, ws, P, round_no[0], device) if ws > 1 else q[:s_done]
    T_all = ctx.trace_prefix(q_all)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    ms_dev = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - n0
    prof = ctx.profile_report()
    autotune = prof.pop("_autotune", {})
    ctx.profile_enable(False)
    ms_max = max_over_ranks(ws, ms_dev, device)
    rhs = sum(s["rhs_solved"] for s in stats)
    value = ws * rhs / (ms_max / 1e3)
    iters = sum(s["iterations_total"] for s in stats)
    updates = sum(s["reliable_updates"] for s in stats)
    max_res = max(s["max_true_residual"] for s in stats)

    # end to end through the C ABI with host buffers: links from pinned host memory, T back to host
    e2e_steps = 0 if args.no_e2e else max(1, min(2, args.steps))
    if e2e_steps:   # untimed warm-up: the library's one-time device buffer for host-resident links
        step(next_first(), links_host)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_rhs = 0
    h2d = d2h = 0
    for _ in range(e2e_steps):
        first = next_first()
        e2e_rhs += step(first, links_host)["rhs_solved"]
        h2d += V * 72 * 8 + 16 * first          # links, earlier quadratures
        d2h += 2 * 16 * (first + P)             # quadratures and prefix estimates
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(ws, time.perf_counter() - t0, device)
    e2e = None
    if e2e_steps:
        e2e = {"value": ws * e2e_rhs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d / e2e_steps),
               "d2h_bytes_per_step": int(d2h / e2e_steps), "steps": e2e_steps}
        # the copy rate of the links from pinned host memory (for reference: the library reads them
        # in place): the first copy after the e2e steps, the same copy repeated at once, and after 2 s
        # of idle host link
        scratch = torch.empty_like(links_dev)
        torch.cuda.synchronize()
        rates = []
        for _ in range(2):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            scratch.copy_(links_host, non_blocking=True)
            c1.record(stream)
            torch.cuda.synchronize()
            rates.append(links_host.numel() * 8 / (c0.elapsed_time(c1) / 1e3) / 1e9)
        time.sleep(2.0)   # the same copy after the host link has been idle for 2 s
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        scratch.copy_(links_host, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        rates.append(links_host.numel() * 8 / (c0.elapsed_time(c1) / 1e3) / 1e9)
        e2e["links_h2d_GBps_after_solve"], e2e["links_h2d_GBps_repeated"], e2e["links_h2d_GBps_after_2s_idle"] = rates
        e2e["host_links"] = "pinned; read in place by the library's link conversion (no staging copy)"
        del scratch

    # plain FP64 solver on the same GPU (one probe = 12 solves), for the mixed-vs-FP64 ratio
    fp64 = None
    if not args.no_fp64:
        first = next_first()
        step(first, links_dev, precision="fp64", probes=1, rhs_block=12)   # warm-up (allocation)
        first += 1
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = step(first, links_dev, precision="fp64", probes=args.fp64_probes, rhs_block=12)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(ws, e0.elapsed_time(e1), device)
        fp64 = {"solves_per_s": ws * st64["rhs_solved"] / (ms64 / 1e3), "rhs": st64["rhs_solved"],
                "iters_per_solve": st64["iterations_total"] / max(1, st64["rhs_solved"]),
                "max_true_residual": st64["max_true_residual"]}

    # stencil alone (Dslash GB/s) in the iteration precision and in FP64
    peak, peak_kind = hbm_peak()
    dslash = None
    if not args.no_dslash:
        op = ctx.make_operator(hprobe.OP_WILSON, 0.0, KAPPA, links_dev, None, csw=args.csw)
        ds = ctx.dslash_bench(op, DIMS, prec, args.rhs_block, 20)
        ds64 = ctx.dslash_bench(op, DIMS, "fp64", 1, 5)
        dslash = {"precision": prec, "nrhs": args.rhs_block, "ms": ds["ms"], "GBps": ds["bytes"] / ds["ms"] / 1e6,
                  "frac_of_%s_hbm" % peak_kind: ds["bytes"] / ds["ms"] / 1e6 / peak,
                  "TFLOPs": ds["flops"] / ds["ms"] / 1e9,
                  "fp64": {"nrhs": 1, "ms": ds64["ms"], "GBps": ds64["bytes"] / ds64["ms"] / 1e6,
                           "TFLOPs": ds64["flops"] / ds64["ms"] / 1e9}}

    # roofline of the dominant kernel of the timed steps (event-timed launches, algorithmic bytes)
    counts = {"rhs_iters": iters, "updates": updates, "exact": updates + (rhs if args.even_odd and prec == "fp64" else 0),
              "groups": sum(s["group_updates"] for s in stats), "eo": bool(args.even_odd), "clover": bool(args.csw)}
    kernels = {}
    for name, rec in prof.items():
        b = kernel_bytes(name, prec, V, dict(counts, launches=rec["launches"]))
        kernels[name] = {"launches": rec["launches"], "ms": rec["ms"],
                         "GBps": (b / (rec["ms"] / 1e3) / 1e9) if b and rec["ms"] > 0 else None}
    tot_ms = sum(r["ms"] for r in prof.values()) or 1.0
    for k in kernels.values():
        k["share"] = k["ms"] / tot_ms
    top = max(kernels.items(), key=lambda kv: kv[1]["ms"])
    top_name, top_rec = top
    top_bytes = kernel_bytes(top_name, prec, V, dict(counts, launches=top_rec["launches"]))
    achieved = top_bytes / (top_rec["ms"] / 1e3) / 1e9 if top_bytes else None
    trace_ncu = None
    nt = NCU_TRAFFIC.get((top_name, source_hash(top_name)))
    if nt and top_bytes and DIMS == (32, 32, 32, 64) and args.rhs_block == 24 and not args.csw:
        # the capture's traffic per byte of algorithmic work, applied to this run's average launch
        trace_ncu = nt["bytes_all_slots"] / nt["alg_bytes_all_slots"] * top_bytes / top_rec["launches"]
    roofline = {"kernel": top_name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": (top_bytes / top_rec["launches"]) if top_bytes else None,
                "mean_launch_ms": top_rec["ms"] / top_rec["launches"],
                "traffic": trace_ncu}

    # the same kernel against the FP32 arithmetic peak: the even-odd stencils of the mixed iteration
    # keep the FP32 FMA pipe busy (binary16 storage, FP32 arithmetic; ncu: pipe_fmaheavy ~65 %), so
    # their ALU roofline is the FP32 rate: 152 SMs x 128 lanes x 2 flop x the SM clock under load
    roof_fp32 = None
    if top_name == "k_eo_even" and prec in ("fp16", "bf16", "fp32"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.get("sm_mhz") or 2070.0
        peak_tf = sms * 128 * 2 * mhz * 1e6 / 1e12
        flops = (V // 2) * 1320 * 2 * iters   # the hop of every even site, V and T steps, per right-hand side
        ach = flops / (top_rec["ms"] / 1e3) / 1e12
        roof_fp32 = {"kernel": top_name, "bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": ach / peak_tf, "flops_per_site_rhs": 1320,
                     "peak_source": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (median SM clock of the timed steps)"
                                    % (sms, mhz)}

    cpu = None   # (the oracle's clover term is a per-site Python loop: no sampled baseline with --csw)
    if rank == 0 and not args.no_cpu_baseline and ws == 1 and not args.csw:
        cpu = cpu_baseline(FP64_ITERS_PER_SOLVE)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math",
                  "fp64": "f64"}[prec] + " + f64 reliable updates",
        "data": "synthetic: SU(3) links exp(i eps H), seeded (no gauge ensemble available)",
        "config": {"workload": "%s %s, kappa 0.12, eps 0.4, %d probes x 12 dilutions per step, "
                               "BiCGStab %s%s, tol 1e-10" % ("x".join(map(str, DIMS)),
                                                              "Clover-Wilson (c_sw %g)" % args.csw if args.csw
                                                              else "Wilson-Dirac", P, prec,
                                                              " on the even-odd Schur complement"
                                                              if args.even_odd else ""),
                   "csw": args.csw,
                   "even_odd": bool(args.even_odd),
                   "lattice": list(DIMS), "probes_per_step": P, "rhs_per_step": 12 * P, "rhs_block": args.rhs_block,
                   "precision": prec, "tol": TOL, "l2": "inputs larger than L2 (each field >= 100 MB)",
                   "eo_kernel": args.eo_kernel, "rhs_per_thread": args.rhs_per_thread, "use_graph": args.use_graph,
                   "parallelism": "dp%d over probe blocks" % ws},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "roofline_fp32": roof_fp32,
        "cpu_baseline": cpu,
        "solver": {"rhs": rhs, "iters_per_solve": iters / max(1, rhs), "reliable_updates_per_solve": updates / max(1, rhs),
                   "max_true_residual": max_res},
        "trace": {"s": int(s_done), "T_s": [float(T_all[-1].real), float(T_all[-1].imag)],
                  "gathered_over_ranks": ws > 1},
        "fp64_solver": fp64,
        "mixed_over_fp64": (value / ws / fp64["solves_per_s"] * ws) if fp64 else None,
        "dslash": dslash,
        "kernels": kernels,
        "autotune": autotune,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle
def oracle_iteration_time(U, reps):
    """Time per iteration of the oracle's BiCGStab (oracle.solvers.bicgstab, unchanged) on one
    right-hand side, stopped after `reps` iterations by its own maxiter."""
    from oracle import operators as O
    from oracle import solvers as S

    V = U.shape[0]
    b = np.zeros((V, 4, 3), dtype=complex)
    b[:, 0, 0] = 1.0             # a probing source h_0 (x) e_0; the cost per iteration does not depend on it
    t0 = time.perf_counter()
    try:
        S.bicgstab(lambda v: O.wilson_apply(v, U, DIMS, KAPPA), b, tol=1e-10, maxiter=reps)
    except RuntimeError:
        pass
    return (time.perf_counter() - t0) / reps


def _links_device():
    try:
        import torch

        return "cuda:0" if torch.cuda.is_available() else "cpu"
    except ImportError:
        return "cpu"


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def _oracle_worker(path, reps, out_q):
    """One host core: the oracle's BiCGStab iterations on the shared links (memory-mapped)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    U = np.load(path, mmap_mode="r")
    out_q.put(oracle_iteration_time(np.asarray(U), reps))


def oracle_all_cores(U, reps=1, workers=None):
    """The oracle on every host core at once: one process per core, each running `reps` BiCGStab
    iterations on its own right-hand side (the links shared through a memory-mapped file); returns
    (seconds per iteration of the slowest worker, workers)."""
    import multiprocessing as mp
    import tempfile

    n = workers or os.cpu_count() or 1
    d = "/dev/shm" if os.path.isdir("/dev/shm") else None
    with tempfile.NamedTemporaryFile(suffix=".npy", dir=d, delete=False) as f:
        path = f.name
    try:
        np.save(path, np.ascontiguousarray(U))
        ctx = mp.get_context("spawn")   # a fork after CUDA initialisation would hang
        q = ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(path, reps, q)) for _ in range(n)]
        for p in procs:
            p.start()
        times = []
        t0 = time.time()
        while len(times) < n:
            try:
                times.append(q.get(timeout=5))
            except Exception:
                dead = [p for p in procs if p.exitcode not in (None, 0)]
                if dead or time.time() - t0 > 1800:
                    for p in procs:
                        if p.is_alive():
                            p.terminate()
                    raise RuntimeError("oracle worker failed (exit codes %s)" % [p.exitcode for p in procs])
        for p in procs:
            p.join(timeout=60)
        return max(times), n
    finally:
        os.unlink(path)


def cpu_baseline(iters_per_solve, reps=2):
    from paper_1302_4018_gb300 import synth

    U = synth.gauge_links(DIMS, EPS, LINK_SEED, device=_links_device())
    n_it = iters_per_solve or FP64_ITERS_PER_SOLVE or 100.0
    nproc, model = host_cpu()
    t_it = oracle_iteration_time(U, reps)
    t_all, n = oracle_all_cores(U, 1)
    return {"value": n / (t_all * n_it), "unit": UNIT, "cores": n, "kind": "oracle",
            "host": {"nproc": nproc, "cpu_model": model},
            "single_thread": {"value": 1.0 / (t_it * n_it), "unit": UNIT, "cores": 1, "s_per_iteration": t_it},
            "sample": "the oracle's BiCGStab (2 Wilson applications per iteration, numpy FP64) on the 32^3x64 "
                      "workload: %d processes at once, one right-hand side and one iteration each (%.1f s per "
                      "iteration, slowest process), and one process alone (%d iterations, %.1f s each); both "
                      "extrapolated to %.1f iterations per solve (the FP64 iteration count of this workload)"
                      % (n, t_all, reps, t_it, n_it)}


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    from paper_1302_4018_gb300 import synth

    U = synth.gauge_links(DIMS, EPS, LINK_SEED, device=_links_device())
    n_it = FP64_ITERS_PER_SOLVE or 100.0
    for _ in range(args.warmup):
        oracle_iteration_time(U, 1)
    times = [oracle_iteration_time(U, 1) for _ in range(args.steps)]
    t_it = sum(times) / len(times)
    value = 1.0 / (t_it * n_it)
    sample = ("each step: one oracle BiCGStab iteration (numpy FP64, one thread) on one right-hand side of the "
              "32^3x64 workload; solves/s = 1 / (time per iteration x %.1f iterations per solve)" % n_it)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_it, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "32^3x64 Wilson-Dirac, kappa 0.12, eps 0.4, tol 1e-10", "lattice": list(DIMS)},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ other workloads
def run_batch(args):
    """Uneven batch: 8^4, 12^4, 16^3x32, 24^3x48 with kappa, eps, s from PCG64(3000), one schedule.
    A step solves the next 1/8 of every lattice's probe sequence (all lattices in the same launches)."""
    import torch

    from paper_1302_4018_gb300 import hprobe, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    cfg = synth.batch_config()
    ops, dims_list, keep = [], [], []
    for c in cfg:
        U = synth.gauge_links(c["dims"], c["eps"], c["link_seed"], device="cuda:0")
        L = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
        keep.append(L)
        ops.append(ctx.make_operator(hprobe.OP_WILSON, 0.0, c["kappa"], L, None))
        dims_list.append(c["dims"])
    frac = 8
    blocks = [c["s"] // frac for c in cfg]
    opts = ctx.make_opts(args.precision, z0_seed=3000, use_graph=1, rhs_block=args.rhs_block * 2,
                         even_odd=args.even_odd)

    def one_step():
        outs, st = ctx.trace_inv_batch(ops, dims_list, blocks, TOL, opts)
        return st

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = ctx.launch_count()
    e0.record(stream)
    stats = [one_step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rhs = sum(s["rhs_solved"] for s in stats)
    out = {"metric": "batched probing solves/s (uneven Wilson lattices, mixed precision, 1e-10)",
           "value": rhs / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.precision + " iteration + f64 true residual", "data": "synthetic",
           "config": {"workload": "batch [8^4, 12^4, 16^3x32, 24^3x48], kappa/eps/s from PCG64(3000), "
                                  "probes per step s/8 each, one schedule, CUDA-graph iteration",
                      "lattices": [list(d) for d in dims_list], "kappa": [c["kappa"] for c in cfg],
                      "eps": [c["eps"] for c in cfg], "s": [c["s"] for c in cfg], "probes_per_step": blocks},
           "gpu_launches": ctx.launch_count() - n0,
           "solver": {"rhs": rhs, "iters_per_solve": sum(s["iterations_total"] for s in stats) / max(1, rhs),
                      "max_true_residual": max(s["max_true_residual"] for s in stats)}}
    print(json.dumps(out), flush=True)


def run_grad(args):
    """24^3x48, kappa 0.118, eps 0.3, mu(x) ~ N(0, 0.01): estimate and per-site mass gradient, s = 128."""
    import torch

    from paper_1302_4018_gb300 import hprobe, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    dims = (24, 24, 24, 48)
    U = synth.gauge_links(dims, 0.3, 1005, device="cuda:0")
    links = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    mf = torch.from_numpy(synth.mass_field(dims, 0.01, 5000)).cuda()
    op = ctx.make_operator(hprobe.OP_WILSON, 0.0, 0.118, links, mf)
    s_max = args.grad_probes
    g = torch.zeros(mf.numel(), dtype=torch.float64, device="cuda:0")
    opts = ctx.make_opts(args.precision, z0_seed=5001, rhs_block=args.rhs_block, even_odd=args.even_odd)
    for _ in range(args.warmup):
        ctx.trace_inv_grad(op, dims, s_max, TOL, opts, g)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [ctx.trace_inv_grad(op, dims, s_max, TOL, opts, g) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rhs = sum(r[2]["rhs_solved"] for r in res)
    T, dTdm, st = res[-1]
    out = {"metric": "probing solves/s with the mass-field gradient (24^3x48 Wilson, 1e-10)",
           "value": rhs / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.precision + " iteration + f64 true residual and gradient accumulation", "data": "synthetic",
           "config": {"workload": "24^3x48 Wilson kappa 0.118 eps 0.3, mu ~ N(0, 0.01), s = %d, gradient" % s_max},
           "estimate": {"T_s": T[-1].real, "dT_dm": dTdm, "grad_norm": float(torch.linalg.norm(g))},
           "solver": st}
    print(json.dumps(out), flush=True)


def run_variance(args):
    """Section 5.2 on the 64^3 Laplacian at condition number ~100 (m = 12/99): hierarchical probing,
    Hadamard vectors in natural order (both with z_0 bias removal) and Z_2 noise.  One step = one
    z_0 seed with S vectors of each sequence; the value is CG probing solves/s over the whole
    study, and the JSON carries the spread of T_s over the seeds at the completion points."""
    import torch

    from paper_1302_4018_gb300 import hprobe

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    dims = (64, 64, 64)
    mass = 12.0 / 99.0
    S = args.variance_vectors
    op = ctx.make_operator(hprobe.OP_LAPLACIAN, mass)
    kinds = ("hp", "natural", "z2")
    # exact trace: the periodic Laplacian is diagonal in Fourier space
    k = [2 * np.pi * np.arange(L) / L for L in dims]
    lam = mass + sum(4 * np.sin(kk / 2) ** 2 for kk in np.meshgrid(*k, indexing="ij"))
    exact = float(np.sum(1.0 / lam))

    # the 7 lowest modes (the constant and one wave along each axis, cos and sin), exact
    # eigenvectors of the periodic Laplacian, for the deflated sequence
    n = int(np.prod(dims))
    xs = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]   # x_1 fastest
    modes, lams = [np.full(n, 1.0 / np.sqrt(n))], [mass]
    for j, L in enumerate(dims):
        ph = 2 * np.pi * xs[j] / L
        for f in (np.cos, np.sin):
            modes.append(np.sqrt(2.0 / n) * f(ph))
            lams.append(mass + 4 * np.sin(np.pi / L) ** 2)
    evecs = torch.from_numpy(np.ascontiguousarray(np.stack(modes))).cuda()
    lams = np.array(lams)
    kinds = kinds + ("hp_deflated",)

    def step(seed):
        out, solves = {}, 0
        for kind in kinds:
            opts = ctx.make_opts("fp64", z0_seed=seed, rhs_block=128, probe_kind="hp" if kind == "hp_deflated" else kind)
            if kind == "hp_deflated":
                T, _, st = ctx.trace_inv_deflated(op, dims, evecs, lams, S, 1e-10, opts)
            else:
                T, _, st = ctx.trace_inv(op, dims, S, 1e-10, opts)
            out[kind] = T.real
            solves += st["rhs_solved"]
        return out, solves

    for w in range(args.warmup):
        step(1000 + w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    runs = [step(1 + i) for i in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    solves = sum(r[1] for r in runs)
    points = [s for s in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048) if s <= S]
    study = {}
    for kind in kinds:
        Ts = np.array([r[0][kind] for r in runs])
        study[kind] = {"s": points,
                       "mean_rel_error": [float(abs(Ts[:, s - 1].mean() - exact) / exact) for s in points],
                       "std_over_seeds": [float(Ts[:, s - 1].std(ddof=1)) if len(Ts) > 1 else None for s in points]}
    # the same hierarchical sequence with every quadrature bracketed to 1e-10 (Gauss / Gauss-Radau
    # bounds from the CG coefficients) instead of a 1e-10 residual
    opts = ctx.make_opts("fp64", z0_seed=1, rhs_block=128)
    _, _, st_res = ctx.trace_inv(op, dims, S, 1e-10, opts)
    ctx.trace_inv_bounds(op, dims, S, 1e-10, opts)
    torch.cuda.synchronize()
    e0.record(stream)
    Tb, lo, hi, st_b = ctx.trace_inv_bounds(op, dims, S, 1e-10, opts)
    e1.record(stream)
    torch.cuda.synchronize()
    bounds = {"solves_per_s": st_b["rhs_solved"] / (e0.elapsed_time(e1) / 1e3),
              "iters_per_solve": st_b["iterations_total"] / max(1, st_b["rhs_solved"]),
              "iters_per_solve_residual_stop": st_res["iterations_total"] / max(1, st_res["rhs_solved"]),
              "T_S": float(Tb[-1].real), "T_S_lower": float(lo[-1]), "T_S_upper": float(hi[-1])}
    # the same 7 lowest modes computed by the library (Chebyshev-filtered subspace iteration)
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    lam_lib, V_lib, res_lib = ctx.laplacian_eigs(op, dims, 7, tol=1e-10)
    t_e = time.perf_counter() - t_e
    P_lib = torch.from_numpy(V_lib).cuda()
    overlap = torch.linalg.svdvals(P_lib @ evecs.T).min().item()   # cosine of the largest principal angle
    eigs = {"k": 7, "seconds": t_e, "max_rel_eigenvalue_error": float(np.max(np.abs(lam_lib - lams) / lams)),
            "max_rel_residual": float(res_lib.max()), "min_cos_principal_angle_to_exact": overlap}
    out = {"metric": "probing solves/s, Section 5.2 variance study (64^3 Laplacian, cond ~100, CG 1e-10)",
           "value": solves / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic (shifted periodic Laplacian, exact trace in closed form)",
           "config": {"workload": "64^3 Laplacian m = 12/99, %d vectors of hierarchical probing (plain and with "
                                  "the 7 lowest modes deflated), natural-order Hadamard and Z_2 noise per z_0 seed, "
                                  "%d seeds" % (S, args.steps)},
           "exact_trace": exact, "study": study, "quadrature_bounds": bounds, "laplacian_eigs": eigs}
    print(json.dumps(out), flush=True)


def run_wilson_deflation(args):
    """Deflated probing of the Wilson matrix (the conclusions' next step, on the Wilson operator):
    8^4, kappa 0.124, eps 0.4 (link seed 1004), or 16^4, kappa 0.115, eps 0.3 (link seed 1002);
    the k eigenpairs of gamma_5 D with the smallest |lambda| from hp_wilson_eigs (or, with
    --defl-svd, the k smallest singular triplets of D from hp_wilson_svd), then per z_0 seed S
    probing vectors with full dilution, plain and deflated (the same FP16 even-odd solves, the
    deflated quadratures corrected on the device).  One step = one seed, both estimates; value =
    probing solves/s; the JSON carries the spread of T_s over the seeds for both and the
    eigensolver's time and residuals."""
    import torch

    from paper_1302_4018_gb300 import hprobe, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    L = args.defl_lattice
    dims = (L, L, L, L)
    kappa, eps, link_seed = (0.124, 0.4, 1004) if L == 8 else (0.115, 0.3, 1002)
    k, S, svd = args.defl_k, args.defl_vectors, args.defl_svd
    U = synth.gauge_links(dims, eps, link_seed, device="cuda:0")
    links = torch.from_numpy(U.view(np.float64).reshape(-1)).to("cuda:0")
    del U
    op = ctx.make_operator(hprobe.OP_WILSON, 0.0, kappa, links, None)
    V = int(np.prod(dims))
    ev = torch.zeros((k, V, 4, 3), dtype=torch.complex128, device="cuda:0")
    lv = torch.zeros_like(ev) if svd else None
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    # the triplets' residual is relative to sigma^2: 1e-9 there is about 1e-10 / sigma on Q
    etol = args.defl_tol if args.defl_tol else (1e-9 if svd else 1e-10)
    if svd:
        lam, ev, lv, res = ctx.wilson_svd(op, dims, k, tol=etol, right=ev, left=lv)
    else:
        lam, ev, res = ctx.wilson_eigs(op, dims, k, tol=etol, evecs=ev)
    torch.cuda.synchronize()
    t_e = time.perf_counter() - t_e

    def step(seed):
        opts = ctx.make_opts(args.precision, z0_seed=seed, rhs_block=96, even_odd=1)
        T0, _, s0 = ctx.trace_inv(op, dims, S, 1e-10, opts)
        if svd:
            T1, _, s1 = ctx.trace_inv_deflated_svd(op, dims, ev, lv, lam, S, 1e-10, opts)
        else:
            T1, _, s1 = ctx.trace_inv_deflated(op, dims, ev, lam, S, 1e-10, opts)
        return T0.real, T1.real, s0["rhs_solved"] + s1["rhs_solved"]

    for w in range(args.warmup):
        step(5000 + w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    runs = [step(1 + i) for i in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    solves = sum(r[2] for r in runs)
    points = [s for s in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512) if s <= S]
    T0 = np.array([r[0] for r in runs])
    T1 = np.array([r[1] for r in runs])
    spread = {"s": points,
              "std_plain": [float(T0[:, s - 1].std(ddof=1)) if len(runs) > 1 else None for s in points],
              "std_deflated": [float(T1[:, s - 1].std(ddof=1)) if len(runs) > 1 else None for s in points],
              "mean_plain": [float(T0[:, s - 1].mean()) for s in points],
              "mean_deflated": [float(T1[:, s - 1].mean()) for s in points]}
    modes = "%d singular triplets of D" % k if svd else "%d modes of gamma_5 D" % k
    out = {"metric": "probing solves/s, deflated Wilson probing (%d^4, kappa %g, %s)" % (L, kappa, modes),
           "value": solves / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f16-storage/f32-math + f64 reliable updates" if args.precision == "fp16" else args.precision,
           "data": "synthetic: SU(3) links exp(i eps H), seeded (no gauge ensemble available)",
           "config": {"workload": "%d^4 Wilson-Dirac, kappa %g, eps %g, link seed %d; %d vectors x 12 "
                                  "dilutions per z_0 seed, plain and with the %s deflated; %d seeds"
                                  % (L, kappa, eps, link_seed, S,
                                     ("%d smallest singular triplets of D" if svd else
                                      "%d smallest |lambda| of gamma_5 D") % k, args.steps),
                      "precision": args.precision, "even_odd": True},
           ("wilson_svd" if svd else "wilson_eigs"): {
               "k": k, "tol": etol, "seconds": t_e, "abs_lambda_min": float(np.abs(lam).min()),
               "abs_lambda_max": float(np.abs(lam).max()), "max_rel_residual": float(res.max())},
           "spread_over_seeds": spread}
    print(json.dumps(out), flush=True)


def _laplacian_exact_trace(dims, mass):
    """Tr A^-1 of the shifted periodic Laplacian: A is diagonal in Fourier space."""
    k = [2 * np.pi * np.arange(L) / L for L in dims]
    lam = mass + sum(4 * np.sin(kk / 2) ** 2 for kk in np.meshgrid(*k, indexing="ij"))
    return float(np.sum(1.0 / lam))


def run_config2(args):
    """The 16^4 Wilson-Dirac configuration: kappa 0.115, eps 0.3, link seed 1002, z_0 seed 2002,
    s = 1..512 probing vectors with full dilution (6144 right-hand sides), BiCGStab to 1e-10 in the
    chosen precision on the even-odd Schur complement; one step = the whole sequence in one call."""
    import torch

    from paper_1302_4018_gb300 import hprobe, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    dims = (16, 16, 16, 16)
    U = synth.gauge_links(dims, 0.3, 1002, device="cuda:0")
    links = torch.from_numpy(U.view(np.float64).reshape(-1)).to("cuda:0")
    del U
    op = ctx.make_operator(hprobe.OP_WILSON, 0.0, 0.115, links, None)
    S = args.config2_vectors
    opts = ctx.make_opts(args.precision, z0_seed=2002, rhs_block=args.rhs_block * 4, even_odd=args.even_odd,
                         eo_kernel=args.eo_kernel)
    for _ in range(max(1, args.warmup)):
        ctx.trace_inv(op, dims, 8, 1e-10, opts)
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        T, _, st = ctx.trace_inv(op, dims, S, 1e-10, opts)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    rhs = sum(st["rhs_solved"] for st in stats)
    pts = [s for s in (1, 2, 32, 64, 128, 256, 512, 1024) if s <= S]
    out = {"metric": "probing solves/s (16^4 Wilson, true residual 1e-10, s = 1..%d)" % S,
           "value": rhs / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math",
                     "fp64": "f64"}[args.precision] + " + f64-class true residual",
           "data": "synthetic: SU(3) links exp(i eps H), seeded",
           "config": {"workload": "16^4 Wilson-Dirac, kappa 0.115, eps 0.3, %d probes x 12 dilutions, BiCGStab %s "
                                  "on the even-odd Schur complement, tol 1e-10" % (S, args.precision),
                      "rhs_block": args.rhs_block * 4},
           "clocks": clk,
           "solver": {"rhs": rhs, "iters_per_solve": sum(st["iterations_total"] for st in stats) / max(1, rhs),
                      "max_true_residual": max(st["max_true_residual"] for st in stats)},
           "T_s": {str(s): [float(T[s - 1].real), float(T[s - 1].imag)] for s in pts}}
    print(json.dumps(out), flush=True)


def run_study(args):
    """Sections 5.2 and 5.3 on synthetic data, every solve on the GPU (statistics on the host):
    (a) speed-up ratio R_s = V_stoc / (V_hp(s) s) with jackknife errors over z_0 draws, on the
        16^4 Wilson lattice (kappa 0.115, eps 0.3, link seed 1002), FP16 even-odd BiCGStab to 1e-10,
        full spin-colour dilution;
    (b) convergence of hierarchical probing, natural-order Hadamard and Z_2 noise (one z_0 each,
        Z_2 with its +-2 (Var/s)^{1/2} interval) on the Laplacians of Section 5.2: 64^3 at
        condition ~1e2, 32^4 at ~1e4 and 64 x 128^2 at ~1e6 (m = 4d / (cond - 1));
    (c) the spread of T_s over many z_0 draws of hierarchical probing on the 64^3 Laplacian
        (Section 5.2's 100 draws x 2048 vectors; +-2 sigma intervals).
    value = probing solves/s over the whole study."""
    import torch

    from paper_1302_4018_gb300 import hprobe, study, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    solves = 0
    t_all = time.perf_counter()
    # (a) Wilson speed-up ratio
    dims_w = (16, 16, 16, 16)
    U = synth.gauge_links(dims_w, 0.3, 1002, device="cuda:0")
    links = torch.from_numpy(U.view(np.float64).reshape(-1)).to("cuda:0")
    del U
    opw = ctx.make_operator(hprobe.OP_WILSON, 0.0, 0.115, links, None)
    S_w, n_w = args.study_wilson_vectors, args.study_seeds
    rows = []
    t0 = time.perf_counter()
    for i in range(n_w):
        T, _, st = ctx.trace_inv(opw, dims_w, S_w, 1e-10, ctx.make_opts("fp16", z0_seed=2002 + i, rhs_block=96,
                                                                         even_odd=1))
        rows.append(T)
        solves += st["rhs_solved"]
    t_w = time.perf_counter() - t0
    Tw = np.array(rows)
    R, eR = study.jackknife_speedup(Tw)
    Vh, eV = study.jackknife_variance(Tw)
    pts = [s for s in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024) if s <= S_w]
    wilson = {"lattice": list(dims_w), "kappa": 0.115, "eps": 0.3, "z0_draws": n_w, "vectors": S_w,
              "completion_points": [2, 32, 512], "seconds": t_w,
              "s": pts, "V_hp": [float(Vh[s - 1]) for s in pts], "V_hp_err": [float(eV[s - 1]) for s in pts],
              "R_s": [float(R[s - 1]) for s in pts], "R_s_err": [float(eR[s - 1]) for s in pts],
              "max_R_s": float(np.max(R)), "argmax_s": int(np.argmax(R)) + 1,
              "mean_T": [float(Tw[:, s - 1].real.mean()) for s in pts]}
    del links, opw
    # (b) Laplacian convergence at three condition numbers
    lap = []
    for dims, cond, S in (((64, 64, 64), 1e2, args.study_lap_vectors), ((32, 32, 32, 32), 1e4, args.study_lap_vectors),
                          ((64, 128, 128), 1e6, max(16, args.study_lap_vectors // 4))):
        mass = 4.0 * len(dims) / (cond - 1.0)
        op = ctx.make_operator(hprobe.OP_LAPLACIAN, mass)
        exact = _laplacian_exact_trace(dims, mass)
        rec = {"lattice": list(dims), "mass": mass, "condition": cond, "exact_trace": exact, "vectors": S}
        pts = [s for s in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048) if s <= S]
        t0 = time.perf_counter()
        for kind in ("hp", "natural", "z2"):
            q = np.zeros(S, dtype=np.complex128)
            T, q, st = ctx.trace_inv(op, dims, S, 1e-10, ctx.make_opts("fp64", z0_seed=7, rhs_block=128,
                                                                        probe_kind=kind), q_inout=q)
            solves += st["rhs_solved"]
            rec[kind] = {"rel_error": [float(abs(T[s - 1].real - exact) / exact) for s in pts],
                         "iters_per_solve": st["iterations_total"] / max(1, st["rhs_solved"])}
            if kind == "z2":
                w = study.z2_interval(q.real)
                rec[kind]["rel_interval"] = [float(w[s - 1] / exact) if s > 1 else None for s in pts]
        rec["s"] = pts
        rec["seconds"] = time.perf_counter() - t0
        lap.append(rec)
    # (c) many z_0 draws of hierarchical probing on the 64^3 Laplacian
    dims, mass = (64, 64, 64), 12.0 / 99.0
    op = ctx.make_operator(hprobe.OP_LAPLACIAN, mass)
    exact = _laplacian_exact_trace(dims, mass)
    S_c, n_c = args.study_draw_vectors, args.study_draws
    t0 = time.perf_counter()
    rows = []
    for i in range(n_c):
        T, _, st = ctx.trace_inv(op, dims, S_c, 1e-10, ctx.make_opts("fp64", z0_seed=5000 + i, rhs_block=128))
        rows.append(T.real)
        solves += st["rhs_solved"]
    Tc = np.array(rows)
    pts = [s for s in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048) if s <= S_c]
    draws = {"lattice": list(dims), "mass": mass, "exact_trace": exact, "z0_draws": n_c, "vectors": S_c,
             "seconds": time.perf_counter() - t0, "s": pts,
             "mean_rel_error": [float(abs(Tc[:, s - 1].mean() - exact) / exact) for s in pts],
             "rel_2sigma": [float(2 * Tc[:, s - 1].std(ddof=1) / exact) for s in pts]}
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_all
    out = {"metric": "probing solves/s, Sections 5.2-5.3 variance study (Wilson 16^4 speed-up ratio, Laplacians "
                     "at condition 1e2 / 1e4 / 1e6, z_0 draws)",
           "value": solves / wall, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16-storage/f32-math + f64",
           "data": "synthetic (seeded SU(3) links; shifted periodic Laplacians with closed-form traces)",
           "config": {"workload": "variance study: Wilson 16^4 R_s over %d z_0 x %d vectors; Laplacian convergence "
                                  "64^3 / 32^4 / 64x128^2; %d z_0 x %d vectors on 64^3" % (n_w, S_w, n_c, S_c)},
           "solves": solves, "wilson_speedup": wilson, "laplacian_convergence": lap, "z0_draws": draws}
    print(json.dumps(out), flush=True)


SPARSE_DIMS = (64, 64, 64)
SPARSE_SEED = 4242


def sparse_kernel_bytes(name, n, nnz, c):
    """Algorithmic DRAM bytes of a sparse-CG kernel over the run: the CSR matrix (12 B per entry
    in FP64, 8 B in FP32, 4 B per row pointer) once per launch, every vector of a
    right-hand-side iteration read or written once (8 B per row in FP64, 4 B in FP32).
    c: rhs_iters, exact (true residuals), launches."""
    if name.startswith("k_bcm_"):             # FP32 iteration, FP64 reliable updates
        mat32 = 8 * nnz + 4 * (n + 1)
        return {"k_bcm_ap": mat32 * c["launches"] + 8 * n * c["rhs_iters"],
                "k_bcm_xr": 24 * n * c["rhs_iters"],
                "k_bcm_p": 12 * n * c["rhs_iters"],
                "k_bcm_fold": 24 * n * c["exact"]}.get(name)
    mat = 12 * nnz + 4 * (n + 1)
    if name == "k_btrue_slot":               # r = b - A x, one pass over the matrix per slot
        return (mat + 16 * n) * c["exact"]
    name = name.replace("k_bcg_", "k_cg_")   # the blocked engine's kernels do the same work
    if name == "k_cg_ap":        # q = A p, (p, q)
        return mat * c["launches"] + 16 * n * c["rhs_iters"]
    if name == "k_cg_xr":        # x += a p, r -= a q, (r, r)
        return 48 * n * c["rhs_iters"]
    if name == "k_cg_p":         # p = r + b p
        return 24 * n * c["rhs_iters"]
    if name == "k_cg_true":      # r = b - A x (launches without a slot to update leave at once)
        return (mat + 16 * n) * c["exact"]
    return None


def run_sparse(args):
    """Algorithm 1 and the probing trace on a general sparse matrix: the weighted graph Laplacian
    plus 0.1 I of the periodic 64^3 grid (edge weights U[0.5, 1.5]) with its rows renumbered by a
    seeded permutation, so that the row order carries no lattice structure (n = 262144, 7 entries
    per row).  One step = the hierarchical colouring of the matrix plus FP64 CG to 1e-10 on the
    first S probing vectors (complex vectors: two real solves each)."""
    import torch

    from oracle import solvers as OS
    from oracle import sparse_probing as OSP
    from paper_1302_4018_gb300 import hprobe, synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = hprobe.Context(0, stream=stream.cuda_stream)
    rp, ci, val = synth.grid_matrix(SPARSE_DIMS, SPARSE_SEED, shift=0.1)
    n, nnz = len(rp) - 1, len(ci)
    dev = lambda a: torch.from_numpy(a).to("cuda:0")
    rp_d, ci_d, val_d = dev(rp), dev(ci), dev(val)
    paths_d = torch.zeros((32, n), dtype=torch.int32, device="cuda:0")
    S = args.sparse_vectors

    def step(rp_, ci_, val_, paths_out, seed, ev=None):
        if ev:
            ev[0].record(stream)
        paths, rad = ctx.sparse_coloring(rp_, ci_, 32, paths_out=paths_out)
        if ev:
            ev[1].record(stream)
        T, _, st = ctx.trace_inv_sparse(rp_, ci_, val_, paths, rad, S, TOL,
                                        ctx.make_opts(args.sparse_precision, z0_seed=seed,
                                                      rhs_block=args.sparse_rhs_block, delta=args.sparse_delta))
        return T, st, rad

    for w in range(args.warmup):
        step(rp_d, ci_d, val_d, paths_d, 500 + w)
    ctx.profile_enable(True)
    ctx.profile_report()
    clocks = Clocks(0)
    n0 = ctx.launch_count()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    e0.record(stream)
    runs = [step(rp_d, ci_d, val_d, paths_d, 1 + i, evs[i]) for i in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    colour_ms = sum(ev[0].elapsed_time(ev[1]) for ev in evs) / args.steps
    launches = ctx.launch_count() - n0
    prof = ctx.profile_report()
    prof.pop("_autotune", None)
    ctx.profile_enable(False)
    stats = [r[1] for r in runs]
    rad = runs[-1][2]
    solves = sum(s["rhs_solved"] for s in stats)
    iters = sum(s["iterations_total"] for s in stats)
    exact = sum(s["reliable_updates"] for s in stats)
    value = solves / (ms / 1e3)

    # end to end: host CSR arrays through the C ABI, paths back to the host and in again
    e2e = None
    if not args.no_e2e:
        step(rp, ci, val, None, 900)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_solves = sum(step(rp, ci, val, None, 901 + i)[1]["rhs_solved"] for i in range(max(1, min(2, args.steps))))
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        k = max(1, min(2, args.steps))
        nlev = len(rad)
        e2e = {"value": e2e_solves / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(2 * rp.nbytes + 2 * ci.nbytes + val.nbytes + 4 * nlev * n),
               "d2h_bytes_per_step": int(4 * 32 * n + 32 * S), "steps": k}

    peak, peak_kind = hbm_peak()
    counts = {"rhs_iters": iters, "exact": exact}
    kernels = {}
    for name, rec in prof.items():
        b = sparse_kernel_bytes(name, n, nnz, dict(counts, launches=rec["launches"]))
        kernels[name] = {"launches": rec["launches"], "ms": rec["ms"],
                         "GBps": (b / (rec["ms"] / 1e3) / 1e9) if b and rec["ms"] > 0 else None}
    tot_ms = sum(r["ms"] for r in prof.values()) or 1.0
    for k_ in kernels.values():
        k_["share"] = k_["ms"] / tot_ms
    top_name, top_rec = max(kernels.items(), key=lambda kv: kv[1]["ms"])
    top_bytes = sparse_kernel_bytes(top_name, n, nnz, dict(counts, launches=top_rec["launches"]))
    if top_name == "k_bcg_ap":
        # FP64 multiply-adds bound this kernel on GB300 (2 flops per entry and right-hand side
        # against the nominal 1.25 TFLOP/s FP64 rate; ncu: FP64 pipe 75% busy, DRAM 16%)
        flops = 2.0 * nnz * iters
        achieved = flops / (top_rec["ms"] / 1e3) / 1e12
        roofline = {"kernel": top_name, "bound": "alu", "achieved": achieved, "peak": FP64_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_TFLOPS, "peak_source": "nominal FP64 rate",
                    "flops_per_launch": flops / top_rec["launches"],
                    "hbm_frac_of_%s" % peak_kind: top_bytes / (top_rec["ms"] / 1e3) / 1e9 / peak,
                    "mean_launch_ms": top_rec["ms"] / top_rec["launches"], "traffic": None}
    else:
        achieved = top_bytes / (top_rec["ms"] / 1e3) / 1e9 if top_bytes else None
        roofline = {"kernel": top_name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": (top_bytes / top_rec["launches"]) if top_bytes else None,
                    "mean_launch_ms": top_rec["ms"] / top_rec["launches"], "traffic": None}

    cpu = None
    if not args.no_cpu_baseline:
        # the oracle as it stands: Algorithm 1 on the whole matrix, then its CG (scipy SpMV as the
        # matrix-vector product) on the first probing vector's two real parts
        import scipy.sparse as ssp

        A = ssp.csr_matrix((val, ci, rp), shape=(n, n))
        t0 = time.perf_counter()
        _, _, opaths = OSP.hierarchical_coloring(A)
        t_col = time.perf_counter() - t0
        ph, Pp = OSP.path_phases(opaths, 0, 1, 1)
        from oracle import probing as OP

        w = OP.probe_values(ph, Pp)[0]
        t0 = time.perf_counter()
        for part in (w.real.copy(), w.imag.copy()):
            if np.any(part):
                OS.cg(lambda x: A @ x, part, tol=TOL)
        t_solve = (time.perf_counter() - t0) / 2
        per_step = solves / args.steps
        cpu = {"value": per_step / (t_col + t_solve * per_step), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "Algorithm 1 on the whole matrix (%.1f s) and oracle CG on the two real parts of "
                         "probing vector 0 (%.2f s per solve); value = solves per step / (colouring + "
                         "solves per step x time per solve)" % (t_col, t_solve)}

    out = {"metric": "probing solves/s, Algorithm 1 + CG trace on a general sparse matrix (n = 262144, CG 1e-10)",
           "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.sparse_precision == "fp64" else "f32 iteration + f64 reliable updates",
           "data": "synthetic (weighted graph Laplacian + 0.1 I of a renumbered periodic grid)",
           "config": {"workload": "renumbered 64^3 periodic grid Laplacian + 0.1 I, %d entries, hierarchical "
                                  "colouring + %d probing vectors, CG (%s iteration) to a true residual "
                                  "of 1e-10" % (nnz, S, args.sparse_precision),
                      "n": n, "nnz": nnz, "vectors": S, "rhs_block": args.sparse_rhs_block,
                      "precision": args.sparse_precision,
                      "radices": rad, "l2": "the iteration vectors of one block exceed L2 (4 x %d MB)" % (n * args.sparse_rhs_block * 4 >> 20)},
           "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
           "colouring_ms": colour_ms,
           "solver": {"rhs": solves, "iters_per_solve": iters / max(1, solves),
                      "reliable_updates_per_solve": exact / max(1, solves),
                      "max_true_residual": max(s["max_true_residual"] for s in stats)},
           "estimate": {"T_S": float(runs[-1][0][-1].real)}, "kernels": kernels}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16", choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--probes-per-step", type=int, default=2)
    ap.add_argument("--rhs-block", type=int, default=24)
    ap.add_argument("--fp64-probes", type=int, default=1)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "batch", "grad", "variance", "sparse", "study", "config2",
                             "wilson_deflation"])
    ap.add_argument("--defl-k", type=int, default=48, help="modes of gamma_5 D deflated (wilson_deflation)")
    ap.add_argument("--defl-vectors", type=int, default=64, help="probing vectors per seed (wilson_deflation)")
    ap.add_argument("--defl-lattice", type=int, choices=(8, 16), default=8,
                    help="wilson_deflation lattice: 8 (8^4, kappa 0.124) or 16 (16^4, kappa 0.115)")
    ap.add_argument("--defl-tol", type=float, default=0.0,
                    help="wilson_deflation eigensolver tolerance (0: 1e-9 for triplets, 1e-10 for eigenpairs)")
    ap.add_argument("--defl-svd", action="store_true",
                    help="wilson_deflation: deflate singular triplets of D (hp_wilson_svd) instead of the "
                         "eigenpairs of gamma_5 D")
    ap.add_argument("--config2-vectors", type=int, default=512)
    ap.add_argument("--study-seeds", type=int, default=32, help="z_0 draws of the Wilson speed-up ratio")
    ap.add_argument("--study-wilson-vectors", type=int, default=512)
    ap.add_argument("--study-lap-vectors", type=int, default=1024)
    ap.add_argument("--study-draws", type=int, default=100)
    ap.add_argument("--study-draw-vectors", type=int, default=2048)
    ap.add_argument("--sparse-vectors", type=int, default=128)
    ap.add_argument("--sparse-rhs-block", type=int, default=64)
    ap.add_argument("--sparse-precision", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--sparse-delta", type=float, default=0.0,
                    help="reliable-update threshold of the FP32 iteration (0: the library default 1e-3)")
    ap.add_argument("--variance-vectors", type=int, default=512)
    ap.add_argument("--even-odd", type=int, default=1, help="1: iterate on the odd-site Schur complement")
    ap.add_argument("--grad-probes", type=int, default=128)
    ap.add_argument("--lattice", default=None,
                    help="L1,L2,L3,L4: another lattice for the headline path (profiling small cases; "
                         "not the benchmark workload)")
    ap.add_argument("--csw", type=float, default=0.0,
                    help="clover coefficient of the Clover-Wilson operator (0: plain Wilson, the headline)")
    ap.add_argument("--eo-kernel", type=int, default=0,
                    help="even-odd V / T step kernels (hp_solver_opts.eo_kernel; 0: autotuned)")
    ap.add_argument("--rhs-per-thread", type=int, default=0,
                    help="hp_solver_opts.rhs_per_thread (with --eo-kernel 1: 1 = 12-real links, 101 = 18-real)")
    ap.add_argument("--use-graph", type=int, default=0, help="replay the iteration chunks from CUDA graphs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-dslash", action="store_true")
    args = ap.parse_args()
    if args.lattice:
        global DIMS
        DIMS = tuple(int(v) for v in args.lattice.split(","))
        assert len(DIMS) == 4
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "grad":
        run_grad(args)
    elif args.workload == "variance":
        run_variance(args)
    elif args.workload == "sparse":
        run_sparse(args)
    elif args.workload == "study":
        run_study(args)
    elif args.workload == "config2":
        run_config2(args)
    elif args.workload == "wilson_deflation":
        run_wilson_deflation(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
