"""Benchmark: RK4 propagation of the unfolded driven Bose dimer at N = 1000 on GB300.

One bench step = STEP_RK4 classical RK4 steps (FP64) of the N = 1000 dimer (D = 999 999
Bloch components, Q0 with 18.4 M stored entries) at the stable step size, inputs resident in
HBM.  Reported: RK4 steps/s (whole job), the roofline of the stage kernel, an end-to-end
number through the C-ABI with host buffers, the CPU oracle timed on the host, and side
measurements (FP32 bulk form, GPU assembly seconds, batched instances, adjoint gradient).

--impl reference times the CPU oracle instead (the deliberately slow reference arm).
Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the data path.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BENCH = 1000
STEP_RK4 = 2000          # RK4 steps per bench step
METRIC = "RK4 steps/s & SpMV HBM GB/s at N=1000; Q/K assembly s; batched/adjoint vs plain"
UNIT = "RK4 steps/s"
PROFILE_JSON = os.path.join(ROOT, "profiles", "rk4_stage_fp64_n1000.json")
# stage kernel of each variant of the library (chosen per context by timing; {f}: Q1 folded into
# slot 0, {c}: 16-bit columns); variant 3 is launched with programmatic dependent launch
KERNEL_OF_VARIANT = {0: "k_stage{b}<S,18,{f},{c}>", 1: "k_stage_pf<S,18,{t},{f},{c}>",
                     2: "k_stage_r2<S,18,{t},{f}>", 3: "k_stage_pdl<S,18,{t},{f},{c}>"}


def kernel_name(info, p):
    """Stage kernel in use for precision slot p (0: FP64, 1: FP32) after the variant timer ran."""
    v = info.rk4_variant[p]
    return KERNEL_OF_VARIANT.get(v, "?").format(b="64" if p == 0 else "32", t="double" if p == 0 else "float",
                                                f="true" if info.q1_folded else "false",
                                                c="true" if info.rk4_compact[p] else "false")


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, max clock, throttle reasons)."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def code_text(src):
    """Source text without comments and blank space, so that a comment edit keeps the hash."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def src_hash():
    """Hash of the stage-kernel sources (code only) that keys the committed DRAM capture."""
    h = hashlib.sha256()
    for f in ("rk4.cu", "stage.cuh", "hyb.cu", "common.cuh"):
        h.update(code_text(open(os.path.join(ROOT, "paper_1812_11626_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def stage_bytes(nnz0, nnz1, D, precision, q1_folded=False, wide_entries=None):
    """Compulsory bytes per RK4 stage launch, averaged over the 4 stages of a step.

    Matrix stream: value + int32 column per stored entry of [Q0 + E Q1 | K] (no row pointers in
    the ELL layout) and of Q1; with Q1 folded into the first slot of its row, one Q1 value per
    row instead.  With 16-bit columns (wide_entries given: the entries still read with int32
    columns, i.e. the long rows' entries and the slots of the escaped rows), value + 2 bytes
    per entry and 2 more per wide entry.  Vectors, per step: stage 1 reads v once (also the
    gather source) and writes y2 and acc; stages 2-3 gather y, read v, write y_next, read+write
    acc; stage 4 gathers y4, reads+writes v, reads acc: 17 vector passes of D elements, plus the
    FP64 master update (read+write) of the FP32 form.
    """
    vb = 8 if precision == 64 else 4
    cols = 4 * nnz0 if wide_entries is None else 2 * nnz0 + 2 * wide_entries
    mat = vb * nnz0 + cols + (vb * D if q1_folded else (vb + 4) * nnz1)
    vec = 17 * vb * D + (16 * D if precision == 32 else 0)
    return (4 * mat + vec) / 4.0


def stage_fp64_ops(nnz0, D, n_long, q1_folded):
    """FP64 operations per FP64 stage launch, averaged over the 4 stages of a step: one FMA per
    stored entry of [Q0 + E Q1 | K], one per short row for the folded Q1 value, 1.75 per row in
    the stage updates (1, 2, 2, 2), and the 2 x 5 shuffle additions of the two warp sums of
    each long row (32 lanes each)."""
    return nnz0 + ((D - n_long) if q1_folded else 0) + 1.75 * D + 2 * 5 * 32 * n_long


def fp64_peak_gops(sm_mhz):
    """FP64 operations per second of GB300 at an SM clock: 152 SMs x 2 per clock (the nominal
    1.25 TFLOP/s counts an FMA as 2 flops at the 2070 MHz maximum)."""
    return 152 * 2 * sm_mhz * 1e6 / 1e9


def wide_entries(info, p):
    """Entries read with int32 columns when the stage kernel in use for precision slot p reads
    the 16-bit columns (None: it reads int32 columns only): the long rows' entries and every
    slot of the escaped rows."""
    if not info.rk4_compact[p]:
        return None
    return info.tail_nnz + info.compact_escaped_rows * info.ell_width_q0


def launches_per_call(n):
    """Kernels one gksl_propagate(n steps, FP64) launches: 4 per step, a step-base setter per
    64-step graph chunk and per remainder, the drive table and the final finiteness check."""
    return 4 * n + (n // 64) + (1 if n % 64 else 0) + 2


# ---------------------------------------------------------------------- reference arm (CPU oracle)

def run_reference(args, rank, world):
    if rank != 0:
        return
    import scipy.sparse  # noqa: F401
    from oracle import native, system as SYS
    from paper_1812_11626_gb300 import workloads as W
    native.build()
    d = W.dimer(N_BENCH)
    t0 = time.perf_counter()
    u = SYS.unfold_dimer(d)
    asm_s = time.perf_counter() - t0
    p = d.params
    Q0 = u.q0(p["J"], p["U"], d.rate)
    K = d.rate * u.K1
    spp = stable_spp_estimate(d)
    h = 2 * np.pi / p["omega"] / spp
    v = SYS.initial_v(d)
    sysc = native.Rk4System(Q0, u.Q1, K, len(v))
    threads = native.rk4_threads()
    sample = 32   # RK4 steps per bench step of the reference arm (bounded sample)
    n = 0
    for _ in range(args.warmup):
        v, _ = sysc.run(p["E"], p["A"], p["omega"], v, h, sample, t0=n * h)
        n += sample
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, _ = sysc.run(p["E"], p["A"], p["omega"], v, h, sample, t0=n * h)
        n += sample
    el = time.perf_counter() - t0
    val = args.steps * sample / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "driven Bose dimer N=1000 (D=999999), FP64 RK4 at the stable step", "N": N_BENCH,
                       "rk4_steps_per_bench_step": sample, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} RK4 steps per bench step (the oracle's C RK4 on {threads} OpenMP "
                                       f"threads); oracle assembly {asm_s:.1f} s untimed"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_assembly_s": asm_s}
    print(json.dumps(line), flush=True)


def stable_spp_estimate(d):
    """Host-only copy of the library's stability bound (used only by the reference arm)."""
    H = (d.params["J"] * d.HJ.to_scipy() + d.params["U"] * d.HU.to_scipy()).toarray()
    H1 = np.diag(d.H1.to_scipy().diagonal().real)
    spread = 0.0
    for e in (d.params["E"] - d.params["A"], d.params["E"] + d.params["A"]):
        M = H + e * H1
        c = np.real(np.diag(M))
        r = np.abs(M).sum(1) - np.abs(np.diag(M))
        spread = max(spread, (c + r).max() - (c - r).min())
    L = np.abs(d.L.to_scipy().toarray())
    diss = 2 * d.rate * L.sum(0).max() * L.sum(1).max()
    return int(np.ceil(2 * np.pi / d.params["omega"] * (spread + diss) / 2.6))


# ---------------------------------------------------------------------- GPU arm

def cpu_baseline_sample():
    """The oracle as it stands on this host: its assembly, then bounded samples of RK4 steps with
    the threaded C RK4 on every host core (about 10 s) and, for context, with scipy's CSR product
    on one thread (about 5 s)."""
    from oracle import native, propagate as OP, system as SYS
    from paper_1812_11626_gb300 import workloads as W
    native.build()
    d = W.dimer(N_BENCH)
    t0 = time.perf_counter()
    u = SYS.unfold_dimer(d)
    asm_s = time.perf_counter() - t0
    p = d.params
    Q0 = u.q0(p["J"], p["U"], d.rate)
    K = d.rate * u.K1
    spp = stable_spp_estimate(d)
    h = 2 * np.pi / p["omega"] / spp
    v = SYS.initial_v(d)
    sysc = native.Rk4System(Q0, u.Q1, K, len(v))
    threads = native.rk4_threads()
    n, el = 0, 0.0
    t0 = time.perf_counter()
    while n < 16 or el < 10.0:
        v, _ = sysc.run(p["E"], p["A"], p["omega"], v, h, 8, t0=n * h)
        n += 8
        el = time.perf_counter() - t0
    value = n / el
    # one thread, scipy
    v1 = SYS.initial_v(d)
    eps = OP.eps_fn(p["E"], p["A"], p["omega"])
    n1, el1 = 0, 0.0
    t0 = time.perf_counter()
    while n1 < 8 or el1 < 5.0:
        v1, _ = OP.rk4(Q0, u.Q1, K, eps, v1, h, 4, t0=n1 * h)
        n1 += 4
        el1 = time.perf_counter() - t0
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} FP64 RK4 steps of the N=1000 dimer (the oracle's C RK4, rows shared over {threads} "
                      f"OpenMP threads), after the oracle's definition-route assembly ({asm_s:.1f} s)",
            "single_thread": {"value": n1 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} steps with scipy's CSR product on one thread"},
            "assembly_s": asm_s}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="profiling case for ncu: N=1000 assembly, then 50 FP64 and 50 FP32 RK4 steps")
    ap.add_argument("--profile-mf", action="store_true",
                    help="profiling case for ncu: the N=1000 matrix-free form, 20 FP64 and 20 FP32 RK4 steps")
    ap.add_argument("--profile-adjoint-small", action="store_true",
                    help="profiling case for ncu: the FP64 adjoint at N=200 over one period of 64 steps")
    ap.add_argument("--profile-block", action="store_true",
                    help="profiling case for ncu: the N=10 workload, 10 periods of 200 FP64 steps on one block")
    ap.add_argument("--profile-adjoint-small-fp32", action="store_true",
                    help="profiling case for ncu: the same with the FP32 adjoint (its wide reverse stages)")
    ap.add_argument("--profile-dense", action="store_true",
                    help="profiling case for ncu: assembly of a dense L at N=100 (the dense dissipator route)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="profiling case for ncu: the 256-instance batch, 40 steps per group")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="profiling case for ncu: one FP64 adjoint gradient of the N=1000 dimer over a "
                         "period of 64 stable steps (drive frequency raised accordingly)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile:
        run_profile_case()
        return
    if args.profile_dense:
        run_profile_dense()
        return
    if args.profile_adjoint_small:
        run_profile_adjoint(200)
        return
    if args.profile_block:
        run_profile_block()
        return
    if args.profile_adjoint_small_fp32:
        run_profile_adjoint(200, 32)
        return
    if args.profile_batch:
        run_profile_batch()
        return
    if args.profile_mf:
        run_profile_mf()
        return
    if args.profile_adjoint:
        run_profile_adjoint()
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl as G
    from paper_1812_11626_gb300 import replicas as R
    from paper_1812_11626_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.Stream()
    d = W.dimer(N_BENCH)
    ctx = G.dimer_context(d, device=local, stream=stream.cuda_stream, flags=G.GKSL_ASM_FP32, assemble=False)
    asm_s = G.gksl_assemble(ctx, G.GKSL_ASM_FP32)
    G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
    info = G.gksl_get_info(ctx)
    D = info.D
    spp = G.gksl_min_stable_steps(ctx)

    def step(prec=64):
        G.gksl_propagate(ctx, spp, STEP_RK4, prec, 0, 0, None)

    # measured rates of this GPU (self-checking probes), outside the timed region
    fma_rate, l2_rate = G.gksl_measure_rates(local)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    # every rank runs its own replica: RK4 steps of all ranks over the slowest rank's time
    ms_all, total_steps = R.reduce_timing(ms, args.steps * STEP_RK4, dist, "cuda")
    value = total_steps / (ms_all * 1e-3)
    avg_launch_ms = ms / (args.steps * STEP_RK4 * 4)
    info = G.gksl_get_info(ctx)   # with the stage kernel chosen at the first propagation
    bytes_launch = stage_bytes(info.nnz_q0, info.nnz_q1, D, 64, bool(info.q1_folded), wide_entries(info, 0))
    hbm, peak_kind = peaks()
    achieved = bytes_launch / (avg_launch_ms * 1e-3) / 1e9
    variant = info.rk4_variant[0]
    kernel = kernel_name(info, 0)
    traffic = None
    if os.path.exists(PROFILE_JSON):
        pj = json.load(open(PROFILE_JSON))
        if pj.get("src_hash") == src_hash():
            key = f"{variant}{'c' if info.rk4_compact[0] else ''}"
            traffic = pj.get("variants", {}).get(key, {}).get("dram_bytes_per_launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_launch,
                "kernel": kernel + " (fused SpMV + RK4 stage update, FP64)"}
    # the co-limit: the FP64 pipe, against its rate at the SM clock sampled in the timed region
    ops = stage_fp64_ops(info.nnz_q0, D, info.long_rows, bool(info.q1_folded))
    fp64_peak = fma_rate / 1e9
    gops = ops / (avg_launch_ms * 1e-3) / 1e9
    roofline["fp64_pipe"] = {"ops_per_launch": ops, "achieved": gops, "peak": fp64_peak, "unit": "G FP64 ops/s",
                             "frac": gops / fp64_peak,
                             "peak_kind": "measured: FP64 FMA chains checked against the host recurrence "
                                          "(gksl_measure_rates), one op per FMA",
                             "derived_peak_at_sampled_clock": fp64_peak_gops(ck["sm_mhz"] if ck else 2070.0)}

    # end to end through the C ABI with pinned host buffers: H2D of v, propagate, D2H of v
    host_in = torch.empty(D, dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(D, dtype=torch.float64, pin_memory=True)
    G.gksl_get_state(ctx, host_in.numpy())
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        G.gksl_set_state(ctx, host_in, 0.0)
        G.gksl_propagate(ctx, spp, STEP_RK4, 64, 0, STEP_RK4, host_out)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e = {"value": R.throughput(1e3 * e2e_s, args.steps * STEP_RK4, dist, "cuda"), "unit": UNIT,
           "h2d_bytes_per_step": 8 * D,
           "d2h_bytes_per_step": 8 * D}

    extras = {}
    if not args.no_extras and rank == 0:
        # FP32 bulk form on the same workload
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        G.gksl_propagate(ctx, spp, STEP_RK4, 32, 0, 0, None)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            G.gksl_propagate(ctx, spp, STEP_RK4, 32, 0, 0, None)
        f1.record(stream)
        torch.cuda.synchronize()
        ms32 = f0.elapsed_time(f1)
        info = G.gksl_get_info(ctx)
        b32 = stage_bytes(info.nnz_q0, info.nnz_q1, D, 32, bool(info.q1_folded), wide_entries(info, 1))
        extras["fp32_bulk"] = {"value": args.steps * STEP_RK4 / (ms32 * 1e-3), "unit": UNIT,
                               "kernel": kernel_name(info, 1), "algorithmic_bytes_per_launch": b32,
                               "achieved_gbs": b32 / (ms32 * 1e-3 / (args.steps * STEP_RK4 * 4)) / 1e9}
        # its error against the FP64 path after STEP_RK4 steps from rho0
        v32, v64 = np.zeros((1, D)), np.zeros((1, D))
        for prec, dst in ((32, v32), (64, v64)):
            G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
            G.gksl_propagate(ctx, spp, STEP_RK4, prec, 0, STEP_RK4, dst)
        o = np.zeros(2)
        G.gksl_observable_diag(ctx, d.obs_diag, np.concatenate([v32, v64]), 2, o)
        extras["fp32_bulk"].update({"steps_compared": STEP_RK4, "max_abs_dv_vs_fp64": float(np.abs(v32 - v64).max()),
                                    "obs_n1_minus_n2_diff_vs_fp64": float(abs(o[0] - o[1]))})
        extras["assembly_s"] = asm_s
        extras["nnz_q0"] = info.nnz_q0
        extras["device_bytes"] = info.device_bytes
        extras["spmv_hbm_gbs"] = achieved
        extras["steps_per_period_stable"] = spp
        tinfo = G.gksl_get_info(ctx)
        extras["stage_kernel_variant"] = {
            p: {"chosen": tinfo.rk4_variant[i], "columns": 16 if tinfo.rk4_compact[i] else 32,
                "timed_us_per_step": [round(x, 2) for x in tinfo.rk4_variant_us[i]],
                "timed_us_per_step_16bit_columns": [round(x, 2) for x in tinfo.rk4_variant_us_c16[i]]}
            for i, p in enumerate(("fp64", "fp32"))}
        extras["stage_columns_16bit"] = {"escaped_rows": tinfo.compact_escaped_rows, "long_rows": tinfo.long_rows,
                                         "long_row_entries": tinfo.tail_nnz}
        # the FP32 stage against HBM by its own bytes: the form in use (timed above), and the fastest
        # variant of each column width as the variant timer measured it (8-step graphs, warm)
        extras["fp32_bulk"]["frac_of_hbm"] = extras["fp32_bulk"]["achieved_gbs"] / hbm
        by_form = {}
        for name, us, wide in (("32-bit columns", tinfo.rk4_variant_us[1], None),
                               ("16-bit columns", tinfo.rk4_variant_us_c16[1],
                                tinfo.tail_nnz + tinfo.compact_escaped_rows * tinfo.ell_width_q0)):
            timed = [(x, v) for v, x in enumerate(us) if x > 0]
            if not timed:
                continue
            t_us, var = min(timed)
            b = stage_bytes(tinfo.nnz_q0, tinfo.nnz_q1, D, 32, bool(tinfo.q1_folded), wide)
            gbs = 4 * b / (t_us * 1e-6) / 1e9
            by_form[name] = {"variant": var, "us_per_step": t_us, "algorithmic_bytes_per_launch": b,
                             "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm}
        extras["fp32_bulk"]["by_column_form"] = by_form
    G.gksl_destroy(ctx)
    if not args.no_extras and rank == 0:
        extras["matrix_free"] = matrix_free_extras(G, W, torch, stream, d, spp, args.steps)
        extras.update(batched_and_adjoint(G, W, torch, l2_rate))
        extras.update(dense_and_asymptotic(G, W, torch))
        extras.update(small_configs(G, W, torch))
        extras["measured_rates"] = {"fp64_fma_per_s": fma_rate, "l2_read_gbs": l2_rate / 1e9,
                                    "how": "gksl_measure_rates: FP64 FMA chains on 4 CTAs per SM checked bit for bit "
                                           "against the host recurrence; 64 passes over a 32 MiB L2-resident buffer "
                                           "read with ld.global.cg, sum checked"}

    if rank == 0:
        cpu = cpu_baseline_sample()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "driven Bose dimer N=1000 (D=999999), FP64 RK4 at the stable step size",
                           "N": N_BENCH, "rk4_steps_per_bench_step": STEP_RK4, "steps_per_period": spp,
                           "l2": "inputs larger than L2 (Q0 stream 233 MB > 129 MB)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": {k: v for k, v in cpu.items() if k != "assembly_s"},
                "e2e": e2e, "gpu_launches": args.steps * launches_per_call(STEP_RK4), "clocks": ck,
                "extras": extras}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def mf_stage_bytes(D, precision):
    """Compulsory bytes per matrix-free stage launch, averaged over the 4 stages of a step: the
    same 17 vector passes as the CSR stages (plus the FP64 master update of the FP32 form) and no
    matrix stream; the O(N) band data and the diagonal of rho are noise at N = 1000."""
    vb = 8 if precision == 64 else 4
    return (17 * vb * D + (16 * D if precision == 32 else 0)) / 4.0


def matrix_free_extras(G, W, torch, stream, d, spp, steps):
    """The matrix-free form (Q applied on the fly) on the same N = 1000 workload: FP64 and FP32
    RK4 steps/s, the bytes it streams, and its distance to the CSR FP64 path after 2000 steps."""
    ctx = G.dimer_context(d, stream=stream.cuda_stream, flags=G.GKSL_ASM_MATRIX_FREE | G.GKSL_ASM_FP32,
                          assemble=False)
    out = {"assembly_s": G.gksl_assemble(ctx, G.GKSL_ASM_MATRIX_FREE | G.GKSL_ASM_FP32)}
    D = d.N * d.N - 1
    out["device_bytes"] = G.gksl_get_info(ctx).device_bytes
    for prec in (64, 32):
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        G.gksl_propagate(ctx, spp, STEP_RK4, prec, 0, 0, None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            G.gksl_propagate(ctx, spp, STEP_RK4, prec, 0, 0, None)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        us_launch = 1e3 * ms / (steps * STEP_RK4 * 4)
        out["fp%d" % prec] = {"value": steps * STEP_RK4 / (ms * 1e-3), "unit": UNIT, "us_per_stage": us_launch,
                              "algorithmic_bytes_per_launch": mf_stage_bytes(D, prec),
                              "achieved_gbs": mf_stage_bytes(D, prec) / (us_launch * 1e-6) / 1e9}
    # distance to the CSR FP64 path after STEP_RK4 FP64 steps from rho0
    ref = G.dimer_context(d, stream=stream.cuda_stream, flags=0)
    va, vb = np.zeros((1, D)), np.zeros((1, D))
    G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
    G.gksl_propagate(ctx, spp, STEP_RK4, 64, 0, STEP_RK4, va)
    G.gksl_propagate(ref, spp, STEP_RK4, 64, 0, STEP_RK4, vb)
    out["max_abs_diff_vs_csr_fp64"] = float(np.abs(va - vb).max())
    G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
    G.gksl_propagate(ctx, spp, STEP_RK4, 32, 0, STEP_RK4, va)
    o = np.zeros(2)
    G.gksl_observable_diag(ref, d.obs_diag, np.concatenate([va, vb]), 2, o)
    out["fp32"]["max_abs_dv_vs_csr_fp64"] = float(np.abs(va - vb).max())
    out["fp32"]["obs_n1_minus_n2_diff_vs_csr_fp64"] = float(abs(o[0] - o[1]))
    G.gksl_destroy(ref)
    G.gksl_destroy(ctx)
    return out


def run_profile_mf():
    """Small, fixed case for ncu: the N = 1000 matrix-free form (vectors only, about 60 MB on the
    device; the 8 MB state vectors fit L2, so DRAM counters read low), 20 FP64 then 20 FP32 steps."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl as G
    from paper_1812_11626_gb300 import workloads as W
    d = W.dimer(N_BENCH)
    ctx = G.dimer_context(d, flags=G.GKSL_ASM_MATRIX_FREE | G.GKSL_ASM_FP32)
    spp = G.gksl_min_stable_steps(ctx)
    G.gksl_propagate(ctx, spp, 20, 64, 0, 0, None)
    G.gksl_propagate(ctx, spp, 20, 32, 0, 0, None)
    print(json.dumps({"profile_case": "matrix-free N=1000", "steps_per_period": spp}), flush=True)
    G.gksl_destroy(ctx)


def run_profile_case():
    """Small, fixed case for ncu: the N = 1000 workload (matrix stream 233 MB > L2, about 1 GB
    held on the device), 50 FP64 then 50 FP32 RK4 steps."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl as G
    from paper_1812_11626_gb300 import workloads as W
    d = W.dimer(N_BENCH)
    ctx = G.dimer_context(d, flags=G.GKSL_ASM_FP32)
    spp = G.gksl_min_stable_steps(ctx)
    G.gksl_propagate(ctx, spp, 50, 64, 0, 0, None)
    G.gksl_propagate(ctx, spp, 50, 32, 0, 0, None)
    info = G.gksl_get_info(ctx)
    print(json.dumps({"profile_case": "N=1000", "nnz_q0": info.nnz_q0, "nnz_q1": info.nnz_q1, "D": info.D,
                      "src_hash": src_hash(), "steps_per_period": spp}), flush=True)
    G.gksl_destroy(ctx)


def run_profile_dense():
    """Small, fixed case for ncu: one assembly of a fully dense L at N = 100, which takes the dense
    dissipator route (k_dense_R twice over the 1e8 entries of R: count, then fill)."""
    import torch
    from paper_1812_11626_gb300 import gksl as G, workloads as W
    N = 100
    ctx = G.gksl_create(N)
    G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=W.random_operator(N, 0.05, 900, hermitian=True))
    G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.02, op=W.random_operator(N, 1.0, 901))
    G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
    sec = G.gksl_assemble(ctx, 0)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "dense L N=100", "assembly_s": sec, "nnz_r": G.gksl_get_info(ctx).nnz_r[0]}),
          flush=True)
    G.gksl_destroy(ctx)


def run_profile_batch():
    """Small, fixed case for ncu: the 256-instance seeded batch (N in {50, 100, 200}), 40 FP32 steps
    per group after the tile autotuning."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl as G
    from paper_1812_11626_gb300 import workloads as W
    b, ctxs, groups = G.dimer_batch(W.batch_instances(256, 1812))
    spps = [spp for _, _, spp in groups]
    sec = G.gksl_batch_propagate(b, spps, [40] * len(groups), 0)
    print(json.dumps({"profile_case": "batch 256", "seconds": sec,
                      "tiles": [G.gksl_batch_info(b, i) for i in range(len(groups))]}), flush=True)
    G.gksl_batch_destroy(b)
    for c in ctxs:
        G.gksl_destroy(c)


def run_profile_block():
    """Small, fixed case for ncu: the N = 10 dimer over its stated 10 periods of 200 FP64 steps,
    v emitted at every period end, so the one-block kernel runs 10 launches of 200 steps."""
    import __graft_entry__
    __graft_entry__.build()
    import numpy as np
    from paper_1812_11626_gb300 import gksl as G
    from paper_1812_11626_gb300 import workloads as W
    d = W.dimer(10)
    ctx = G.dimer_context(d)
    v = np.zeros((10, d.N * d.N - 1))
    t0 = time.perf_counter()
    G.gksl_propagate(ctx, 200, 2000, 64, 0, 200, v)
    el = time.perf_counter() - t0
    print(json.dumps({"profile_case": "block N=10", "seconds": el, "v_last_max": float(np.abs(v[-1]).max())}),
          flush=True)
    G.gksl_destroy(ctx)


def run_profile_adjoint(N=N_BENCH, precision=64):
    """Small, fixed case for ncu: the FP64 (or FP32) adjoint of the N = 1000 dimer (every matrix
    stream larger than L2, about 1.5 GB on the device), or of the N = 200 dimer of the adjoint
    workload, over one period of 64 steps.  The drive frequency is raised so that 64 steps are the stable
    step count (h at the stability bound, as in the full-size runs), which keeps the case short
    without changing any kernel's work per step."""
    import __graft_entry__
    __graft_entry__.build()
    import numpy as np
    from paper_1812_11626_gb300 import gksl as G
    from paper_1812_11626_gb300 import workloads as W
    d = W.dimer(N)
    ctx = G.dimer_context(d)
    spp = G.gksl_min_stable_steps(ctx)
    omega = d.params["omega"] * spp / 64.0
    G.gksl_set_drive(ctx, d.params["E"], d.params["A"], omega)
    G.gksl_assemble(ctx, G.GKSL_ASM_FP32 | G.GKSL_ASM_TRANSPOSE)
    G.gksl_set_rho0(ctx, d.rho0_dense().real.copy(), d.rho0_dense().imag.copy())
    S = G.gksl_min_stable_steps(ctx)
    grad = np.zeros(4)
    t0 = time.perf_counter()
    loss = G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, 1, precision, grad)
    el = time.perf_counter() - t0
    print(json.dumps({"profile_case": f"adjoint N={N} FP{precision}", "steps_per_period": S, "omega": omega,
                      "seconds": el,
                      "loss": loss, "grad": list(grad)}), flush=True)
    G.gksl_destroy(ctx)


def batch_group_bytes(D, B, entries, pair_entries, path, nnz_union):
    """Bytes one FP32 RK4 step of a batched group requests from L1/L2: per stage and instance chunk
    every stored entry's column and values (row paths: 8 B per channel entry; pair path: 4 B of
    column and two float4 of channel values, 36 B, per pair-unit entry), one 4-byte gather per
    entry and instance (channel entries on rows, pair-unit entries on pairs), and the stage
    updates' state traffic (12 + 16 + 16 + 24 B per row and instance over the four stages).
    Returns (requested bytes, algorithmic bytes 4 (16 nnz_union + 12 D B) of the workload
    statement, nnz_union the union pattern of the channels)."""
    if path == 2:
        req = 4 * (36 * pair_entries + 4 * pair_entries * B)
    else:
        req = 4 * (8 * entries + 4 * entries * B)
    req += (12 + 16 + 16 + 24) * D * B
    alg = 4 * (16 * nnz_union + 12 * D * B)
    return req, alg


def batched_and_adjoint(G, W, torch, l2_rate=None):
    """Side measurements: the batched form (256 seeded instances, N in {50, 100, 200}) and the
    adjoint gradient at N = 200 over period 20, each against the plain FP64 single-instance path."""
    out = {}
    inst = W.batch_instances(256, 1812)
    b, ctxs, groups = G.dimer_batch(inst)
    spps = [spp for _, _, spp in groups]
    n_inst = [len(idx) for _, idx, _ in groups]
    groups = {N: idx for N, idx, _ in groups}
    # a tenth of a period per group at its stable step size (the per-step cost is what is timed)
    steps = [max(1, s // 10) for s in spps]
    G.gksl_batch_propagate(b, spps, steps, 0)   # warm-up, includes the tile autotuning
    G.gksl_batch_reset(b)
    sec = G.gksl_batch_propagate(b, spps, steps, 0)
    inst_steps = sum(n * s for n, s in zip(n_inst, steps))
    tiles = [G.gksl_batch_info(b, i) for i in range(len(ctxs))]
    stats = [G.gksl_batch_group_stats(b, i) for i in range(len(ctxs))]
    nnz_union = [G.gksl_get_info(c).nnz_q0 for c in ctxs]   # [Q0 + E Q1 | K] of each group's context
    # error of the batched form (FP32 bulk, FP64 master) against the plain FP64 path: the first
    # instance of every group after the same steps, from the same state
    errors, first = [], 0
    for (N, idx), spp_g, s in zip(sorted(groups.items()), spps, steps):
        x = inst[idx[0]]
        D_g = N * N - 1
        vb = np.zeros(D_g)
        G.gksl_batch_get_state(b, first, vb)
        d1 = W.dimer(N, dict(A=x["A"], gamma=x["gamma"]))
        c1 = G.dimer_context(d1, flags=0)
        vp = np.zeros((1, D_g))
        G.gksl_propagate(c1, spp_g, s, 64, 0, s, vp)
        o = np.zeros(2)
        G.gksl_observable_diag(c1, d1.obs_diag, np.stack([vb, vp[0]]), 2, o)
        errors.append({"N": N, "instance": first, "steps": s, "max_abs_dv": float(np.abs(vb - vp[0]).max()),
                       "obs_n1_minus_n2_diff": float(abs(o[0] - o[1]))})
        G.gksl_destroy(c1)
        first += len(idx)
    G.gksl_batch_destroy(b)
    # plain FP64 single-instance path on the same groups for comparison
    plain = 0.0   # seconds the plain path needs for the same instance-steps, run one by one
    for c, spp_g, s, ni in zip(ctxs, spps, steps, n_inst):
        n = min(s, 2000)
        G.gksl_propagate(c, spp_g, 64, 64, 0, 0, None)   # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.gksl_propagate(c, spp_g, n, 64, 0, 0, None)
        torch.cuda.synchronize()
        plain += (time.perf_counter() - t0) / n * s * ni
    for c in ctxs:
        G.gksl_destroy(c)
    # roofline of the group that bounds the run (the largest N, which runs the most steps): its
    # per-step time alone (the autotuner's CUDA-event timing) against the measured L2 read rate
    gi = len(stats) - 1
    Dg, Bg, Ug, Pg, path = stats[gi]
    l2b, algb = batch_group_bytes(Dg, Bg, Ug, Pg, path, nnz_union[gi])
    us = tiles[gi][1]
    hbm, _ = peaks()
    roof = None
    if us > 0:
        roof = {"bound": "l2", "group_N": sorted(groups)[gi], "rows": Dg, "instances": Bg, "channel_entries": Ug,
                "pair_unit_entries": Pg, "path": ["16-byte rows", "scalar rows", "pair units"][path],
                "us_per_step": us, "requested_bytes_per_step": l2b, "achieved": l2b / (us * 1e-6) / 1e9,
                "peak": (l2_rate / 1e9) if l2_rate else None, "unit": "GB/s",
                "frac": (l2b / (us * 1e-6) / l2_rate) if l2_rate else None,
                "peak_kind": "measured: L2-resident read rate (gksl_measure_rates); achieved counts the bytes the "
                             "kernel requests from L1/L2, some of which L1 serves",
                "algorithmic_bytes_per_step": algb, "algorithmic_gbs": algb / (us * 1e-6) / 1e9,
                "algorithmic_frac_of_hbm": algb / (us * 1e-6) / 1e9 / hbm}
    out["batched"] = {"instance_steps_per_s": inst_steps / sec, "instances": sum(n_inst), "roofline": roof,
                      "groups": {str(N): {"instances": n, "steps": s, "instances_per_lane": t[0], "tuned_us": t[1],
                                          "path": ["16-byte rows", "scalar rows", "pair units"][st[4]]}
                                 for N, n, s, t, st in zip(sorted(groups), n_inst, steps, tiles, stats)},
                      "plain_fp64_instance_steps_per_s": inst_steps / plain if plain > 0 else None,
                      "error_vs_plain_fp64": errors}
    # adjoint at N = 200: gradient of the mean of <n1 - n2> over period 20 at the stable step
    # size (the adjoint workload), FP64 and FP32, against a plain FP64 forward pass
    d = W.dimer(200)
    c = G.dimer_context(d)
    try:
        S = G.gksl_min_stable_steps(c)
        P = 20
        grads = {}
        for prec in (64, 32):
            grad = np.zeros(4)
            t0 = time.perf_counter()
            G.gksl_adjoint_timeavg(c, d.obs_diag, S, P, prec, grad)
            el = time.perf_counter() - t0
            grads[prec] = grad
            out[f"adjoint_fp{prec}"] = {"seconds": el, "periods": P, "steps_per_period": S, "forward_steps": P * S,
                                        "steps_per_s": P * S / el, "grad_A_gamma_J_U": list(grad)}
        out["adjoint_fp32"]["max_rel_diff_vs_fp64"] = float(np.max(np.abs(grads[32] - grads[64]) /
                                                                   np.abs(grads[64])))
        G.gksl_propagate(c, S, 64, 64, 0, 0, None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.gksl_propagate(c, S, S, 64, 0, 0, None)
        torch.cuda.synchronize()
        out["adjoint_plain_fp64_steps_per_s"] = S / (time.perf_counter() - t0)
    finally:
        G.gksl_destroy(c)
    return out


def small_configs(G, W, torch):
    """The small workloads: the N = 10 dimer over its stated 10 periods of 200 steps (v emitted at
    every period end), through the one-block path the library uses at this size and through the
    stage kernels (GKSL_RK4_BLOCK=0), FP64; and the N = 100 dimer's FP64 and FP32 rates over 20 000
    steps at 4 000 steps per period."""
    import numpy as np
    out = {}
    d = W.dimer(10)
    ctx = G.dimer_context(d)
    try:
        D = d.N * d.N - 1
        v = np.zeros((10, D))
        res = {}
        for name, env in (("one block", None), ("stage kernels", "0")):
            old = os.environ.get("GKSL_RK4_BLOCK")
            if env is None:
                os.environ.pop("GKSL_RK4_BLOCK", None)
            else:
                os.environ["GKSL_RK4_BLOCK"] = env
            try:
                best = 1e9
                for _ in range(4):
                    G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
                    t0 = time.perf_counter()
                    G.gksl_propagate(ctx, 200, 2000, 64, 0, 200, v)
                    best = min(best, time.perf_counter() - t0)
            finally:
                if old is None:
                    os.environ.pop("GKSL_RK4_BLOCK", None)
                else:
                    os.environ["GKSL_RK4_BLOCK"] = old
            res[name] = {"seconds": best, "steps_per_s": 2000 / best}
        out["config_n10_fp64_10_periods"] = res
    finally:
        G.gksl_destroy(ctx)
    d = W.dimer(100)
    ctx = G.dimer_context(d)
    try:
        res = {}
        for prec in (64, 32):
            G.gksl_propagate(ctx, 4000, 4000, prec, 0, 0, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.gksl_propagate(ctx, 4000, 20000, prec, 0, 0, None)
            torch.cuda.synchronize()
            res[f"fp{prec}_steps_per_s"] = 20000 / (time.perf_counter() - t0)
        out["config_n100"] = res
    finally:
        G.gksl_destroy(ctx)
    return out


def dense_and_asymptotic(G, W, torch):
    """Side measurements of the general-dissipator and asymptotic-state forms at N = 100:
    assembly of a fully dense L and of a full-rank Kossakowski matrix (the dense route), RK4 on the
    resulting 1e8-entry system, and the bifurcation scan over 32 interactions U with the paper's
    transient of 10 periods."""
    out = {}
    N = 100
    D = N * N - 1
    H = W.random_operator(N, 0.05, 900, hermitian=True)
    H1 = W.CSR.from_dense(np.diag(np.linspace(-1.0, 1.0, N)).astype(complex))
    L = W.random_operator(N, 1.0, 901)
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.set_csr_operator(G.gksl_set_h1, ctx, op=H1)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.02, op=L)
        G.gksl_set_drive(ctx, 0.3, 0.5, 1.0)
        G.gksl_assemble(ctx, 0)                 # warm-up (module loads, allocator)
        G.set_csr_operator(G.gksl_set_dissipator, ctx, 0, 0.02, op=L)
        sec = G.gksl_assemble(ctx, 0)
        info = G.gksl_get_info(ctx)
        re, im = W.random_density_matrix(N, 3, 902)
        G.gksl_set_rho0(ctx, re, im)
        spp = G.gksl_min_stable_steps(ctx)
        G.gksl_propagate(ctx, spp, 16, 64, 0, 0, None)
        torch.cuda.synchronize()
        n = 64
        t0 = time.perf_counter()
        G.gksl_propagate(ctx, spp, n, 64, 0, 0, None)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        stage_bytes_dense = 12 * info.nnz_q0 + 17 * 8 * D / 4.0
        out["dense_L_n100"] = {"assembly_s": sec, "nnz_R": info.nnz_r[0], "nnz_q0_plus_E_q1": info.nnz_q0,
                               "rk4_steps_per_s": n / el,
                               "stage_bytes": stage_bytes_dense, "stage_gbs": stage_bytes_dense * 4 * n / el / 1e9,
                               "route": "dense (the sparse product would have about 5e9 terms)"}
    finally:
        G.gksl_destroy(ctx)
    # full-rank Kossakowski matrix: c 1 + u u^+ (rank D, built in O(D^2) on the host)
    rng = np.random.default_rng(5)
    u = (rng.standard_normal(D) + 1j * rng.standard_normal(D)) / np.sqrt(2 * D)
    A = np.outer(u, u.conj())
    A[np.diag_indices(D)] += 0.05
    ctx = G.gksl_create(N)
    try:
        G.set_csr_operator(G.gksl_set_h0_component, ctx, 0, 1.0, op=H)
        G.gksl_set_drive(ctx, 0.0, 0.0, 1.0)
        t0 = time.perf_counter()
        G.gksl_set_kossakowski(ctx, np.ascontiguousarray(A.real), np.ascontiguousarray(A.imag))
        set_s = time.perf_counter() - t0
        sec = G.gksl_assemble(ctx, 0)
        info = G.gksl_get_info(ctx)
        out["kossakowski_full_rank_n100"] = {"assembly_s": sec, "set_kossakowski_s": set_s,
                                             "nnz_R": info.nnz_r[0], "rank": D}
    finally:
        G.gksl_destroy(ctx)
    del A
    # bifurcation scan: 32 values of U, transient 10 T, one more period for the residual
    U = np.linspace(0.05, 1.0, 32)
    t0 = time.perf_counter()
    pops, spp, res, per = G.bifurcation_scan(N, U, transient=10, max_periods=1)
    el = time.perf_counter() - t0
    out["bifurcation_scan_n100"] = {"U_values": 32, "steps_per_period": spp, "periods": per,
                                    "seconds_incl_assembly": el, "instance_steps_per_s": 32 * per * spp / el,
                                    "max_period_residual": float(res.max()), "min_period_residual": float(res.min())}
    return out


if __name__ == "__main__":
    main()
