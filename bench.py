"""Benchmark: LR-CCSD residual throughput on one GB300 (or N replicas).

One step = the two residual maps that every response iteration applies, on a
batch of right-hand sides (3 dipole components x 4 frequencies):
sigma = A X (Eq. 30) and the transpose product A^T Y (left response,
Eq. 32), at the converged CCSD amplitudes of the synthetic system.
Metric: nominal complex flops per second,
    F_sigma = 8 [R (P_O P_V^2 + O^3 V^3) + P_V^2 L]   per map,
counted once per map regardless of the contraction order or precision scheme.
Alongside: alpha(omega) solves/s of a full lrcc_solve on the same batch.

--impl reference times the CPU oracle (the plain complex128 PyTorch CPU
restatement) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

PREC_NAMES = {"fp64": 0, "tf32": 1, "bf16x3": 2, "fp64emu": 3}
DTYPE_NAMES = {"fp64": "c128 (f64)", "tf32": "tf32 tensor-core + f64", "bf16x3": "bf16x3 tensor-core + f64",
               "fp64emu": "c128 via 7x6-bit integer slices on bf16 tensor cores"}


def nominal_flops(O, V, L, R, assembly=True):
    """F_sigma = 8 [R (P_O P_V^2 + O^3 V^3) + P_V^2 L]; the assembly term is left
    out when the <ab||ef> matrix is cached (it is then built once per context,
    not once per residual map)."""
    po, pv = O * (O - 1) // 2, V * (V - 1) // 2
    return 8.0 * (R * (po * pv * pv + O ** 3 * V ** 3) + (pv * pv * L if assembly else 0))


def recorded_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    when the kernel's source has changed since the counters were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "tc_gemm_traffic_c2.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith("#") or "=" not in line:
            continue
        kv = dict(x.split("=", 1) for x in line.split())
        if kv.get("kernel") != kernel:
            continue
        src = os.path.join(ROOT, kv["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return float(kv["bytes_per_launch"]) if sha == kv.get("sha256_16") else None
    return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        mine = [s for s in self.samples if s and s[0] == os.environ.get("LOCAL_RANK", "0")] or self.samples
        sm = [float(s[1]) for s in mine if len(s) > 2 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in mine if len(s) > 2 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in mine:
            for k, n in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(mine)}


def workload_name(workload, cfg):
    """The workload string both arms report in config.workload."""
    return (f"{workload}: O={cfg['O']} V={cfg['V']} L={cfg['L']}, R={len(cfg['comps']) * len(cfg['omegas'])} RHS "
            f"({len(cfg['comps'])} comps x {len(cfg['omegas'])} omegas), sigma + A^T Y per step")


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """CPU oracle on a bounded sample: sigma = A X for ONE right-hand side of the
    same system (the oracle as it stands, all host cores)."""
    if rank != 0:
        return
    import torch
    from oracle import ccsd
    cfg = synth.CONFIGS[args.workload]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    model = ccsd.build(s)
    x0, _ = ccsd.mp2(model)
    amp = synth.random_amplitudes(cfg["O"], cfg["V"], 1, seed=123, scale=0.05)
    lay = model.lay
    X = lay.join(torch.as_tensor(amp["t1"][0]), torch.as_tensor(amp["t2u"][0]))
    for _ in range(max(0, args.warmup)):
        model.jvp(x0, X)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        model.jvp(x0, X)
        model.vjp(x0, X)
        times.append(time.perf_counter() - t0)
    F = 2 * nominal_flops(cfg["O"], cfg["V"], cfg["L"], 1, assembly=False)
    v = F / statistics.median(times) / 1e12
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": "LR-CCSD residual TFLOP/s", "value": v, "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128 (f64, CPU)", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, cfg),
                       "flop_count": "2 x 8 R (P_O P_V^2 + O^3 V^3) per step; each timed step here is a sample of "
                                     "R = 1 right-hand side, the rate is per the same count"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": "one right-hand side of the workload (the oracle's own sigma and A^T products)"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(cfg):
    """The oracle timed on one right-hand side of the same workload (10-30 s)."""
    import torch
    from oracle import ccsd
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    model = ccsd.build(s)
    x0, _ = ccsd.mp2(model)
    amp = synth.random_amplitudes(cfg["O"], cfg["V"], 1, seed=123, scale=0.05)
    X = model.lay.join(torch.as_tensor(amp["t1"][0]), torch.as_tensor(amp["t2u"][0]))
    t0 = time.perf_counter()
    model.jvp(x0, X)
    model.vjp(x0, X)
    dt = time.perf_counter() - t0
    F = 2 * nominal_flops(cfg["O"], cfg["V"], cfg["L"], 1, assembly=False)
    return {"value": F / dt / 1e12, "unit": "TFLOP/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"sigma + A^T Y for 1 of the {len(cfg['comps']) * len(cfg['omegas'])} right-hand sides "
                      f"({dt:.1f} s)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--prec", default="bf16x3", choices=list(PREC_NAMES))
    ap.add_argument("--solver", default="diis", choices=["diis", "subspace"],
                    help="response/Lambda solver: per right-hand-side DIIS or one shared subspace "
                         "(FP64-class precisions only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--fns", action="store_true",
                    help="FNS++ workload: truncate to the config's 'keep' virtuals, then ground state and alpha")
    ap.add_argument("--profile-csv", default=None,
                    help="write every timed GEMM launch (kernel, M, N, K, batch, ms, flops) to this CSV file")
    ap.add_argument("--ladder-only", action="store_true",
                    help="time only the particle-particle ladder (no ground state); used for kernel profiling")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_2503_23144_gb300 import lrcc as L
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    cfg = synth.CONFIGS[args.workload]
    O, V, Lx = cfg["O"], cfg["V"], cfg["L"]
    comps, omegas = list(cfg["comps"]), list(cfg["omegas"])
    R = len(comps) * len(omegas)
    prec = PREC_NAMES[args.prec]
    s = synth.make_system(O, V, Lx, cfg["seed"])
    opt = L.lrcc_default_options()
    opt.prec = prec
    opt.solver = 1 if args.solver == "subspace" else 0
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V, opt)
    if args.ladder_only:
        return ladder_only(args, L, ctx, O, V, Lx, R, prec, world, rank, local, pg)
    if args.fns:
        return fns_run(args, L, ctx, cfg, rank)
    E, itT, itL = L.lrcc_ccsd_ground(ctx)
    # linearisation point: the converged CCSD amplitudes (read back once, outside timing)
    t_host = L.lrcc_get_amplitudes(ctx, 0)
    n1, n2 = O * V, O * O * V * V
    x_host = np.empty((R, n1 + n2), dtype=np.complex128)
    iu, ju = np.triu_indices(O, 1)
    au, bu = np.triu_indices(V, 1)
    for r in range(R):
        a = synth.random_amplitudes(O, V, 1, seed=2000 + 17 * rank + r, scale=0.05)
        t2 = np.zeros((O, O, V, V), dtype=np.complex128)
        u = a["t2u"][0]
        I, J, A, B = iu[:, None], ju[:, None], au[None, :], bu[None, :]
        t2[I, J, A, B] = u
        t2[J, I, A, B] = -u
        t2[I, J, B, A] = -u
        t2[J, I, B, A] = u
        x_host[r, :n1] = a["t1"][0].reshape(-1)
        x_host[r, n1:] = t2.reshape(-1)
    # the residual hook projects the doubles block onto its antisymmetric part
    dev = torch.device("cuda", local)
    t_dev = torch.as_tensor(t_host).to(dev)
    x_dev = torch.as_tensor(x_host).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # the maps lrcc_solve applies: linearised at the converged T (t = None reuses
    # the primal values the context keeps from lrcc_ccsd_ground)
    def step():
        a = L.lrcc_residual_dev(ctx, L.LRCC_RES_SIGMA, None, x_dev, prec=prec)
        b = L.lrcc_residual_dev(ctx, L.LRCC_RES_VJP, None, x_dev, prec=prec)
        return a, b

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches0 = L.lrcc_kernel_launches(ctx)
    clocks = Clocks()
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    L.lrcc_profile(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (256 MB > 129 MB L2)
        ev[k][0].record()
        step()
        ev[k][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if pg:
        pg.barrier()
    L.lrcc_profile(ctx, False)
    if args.profile_csv:
        L.lrcc_profile_dump(ctx, args.profile_csv)
    ms = [a.elapsed_time(b) for a, b in ev]
    launches = (L.lrcc_kernel_launches(ctx) - launches0) // args.steps
    stats = L.lrcc_kernel_stats(ctx)
    total = sum(ms)
    if pg:
        t = torch.tensor([total], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total = float(t.item())
    # the ladder caches <ab||ef> at this size (c2: 0.6 GB), so no assembly per map
    F_step = 2 * nominal_flops(O, V, Lx, R, assembly=False)
    value = world * F_step * args.steps / (total / 1e3) / 1e12

    # end to end through the host-buffer ABI: H2D of X and T, D2H of both results
    e2e_t = []
    for _ in range(2):
        t0 = time.perf_counter()
        L.lrcc_residual(ctx, L.LRCC_RES_SIGMA, None, x_host, prec=prec)
        L.lrcc_residual(ctx, L.LRCC_RES_VJP, None, x_host, prec=prec)
        e2e_t.append(time.perf_counter() - t0)
    e2e = F_step / min(e2e_t) / 1e12 * world
    h2d = 2 * x_host.nbytes
    d2h = 2 * x_host.nbytes
    clk = clocks.stop()

    # alpha(omega) solves/s: a full lrcc_solve on the same batch (X, F X, Y, alpha)
    solves = None
    if not args.no_solve:
        torch.cuda.synchronize()
        # weak scaling: each rank solves its own frequencies (shifted grid), no exchange
        my_omegas = [w + 1e-3 * rank for w in omegas]
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        alpha, err = L.lrcc_solve(ctx, my_omegas, comps)
        dt = time.perf_counter() - t0
        if pg:
            t = torch.tensor([dt], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            dt = float(t.item())
        n64, nmix = L.lrcc_solve_counts(ctx)
        solves = {"value": world * R / dt, "unit": "alpha(omega)/s", "seconds": dt, "rhs": R,
                  "max_residual": float(err.max()), "precision": args.prec, "solver": args.solver,
                  "alpha_zz_0": float(alpha[0, -1, -1].real), "fp64_maps": n64, "mixed_maps": nmix,
                  "phase_ms": [round(x, 1) for x in L.lrcc_phase_times(ctx)]}

    # roofline of the dominant kernel family in the timed region
    hbm, bf16, bf16s, src = load_peaks()
    dom = max(stats.items(), key=lambda kv: kv[1]["ms"]) if stats else None
    roof = None
    if dom:
        name, st = dom
        achieved = st["flops"] / (st["ms"] / 1e3) / 1e12 / 1.0
        if name == "gemm_tc_bf16x3":
            peak, unit, bound = bf16 / 3.0, "TFLOP/s", "tensor"     # 3 bf16 products per real product
            note = f"bf16 {src} peak / 3 (bf16x3 split); complex flops counted 8 per CMAC"
        elif name == "gemm_tc_f64emu":
            # 28 bf16 slice products (7 diagonals) per real product, 4 real per complex
            peak, unit, bound = bf16 / 28.0, "TFLOP/s", "tensor"
            note = f"bf16 {src} peak / 28 (7x6-bit slices, diagonals 0..6); complex flops counted 8 per CMAC"
        elif name == "gemm_tc_tf32":
            peak, unit, bound = bf16 / 2.0, "TFLOP/s", "tensor"     # tf32 dense = bf16 / 2 nominal
            note = f"bf16 {src} peak x tf32/bf16 nominal ratio 1/2"
        else:
            peak, unit, bound = 1.25, "TFLOP/s", "alu"              # FP64 nominal (FMA pipes)
            note = "GB300 FP64 nominal 1.25 TFLOP/s"
        traffic = recorded_traffic(name) if args.workload == "c2" else None
        roof = {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic, "launches": st["count"],
                "algorithmic_bytes_per_launch": st["bytes"] / max(st["count"], 1),
                "share_of_step": st["ms"] / total, "peak_note": note}

    line = {
        "metric": "LR-CCSD residual TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[args.prec],
        "data": "synthetic",
        "config": {"workload": workload_name(args.workload, cfg),
                   "flops_per_step": F_step, "flop_count": "2 x 8 R (P_O P_V^2 + O^3 V^3); <ab||ef> cached, not counted",
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world} (RHS sharding, no collective)"},
        "e2e": {"value": e2e, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clk, "roofline": roof, "alpha_solves": solves,
        "ground_state": {"E_corr": [E.real, E.imag], "iters_T": itT, "iters_L": itL},
        "kernels": {k: {"count": v["count"], "ms": v["ms"]} for k, v in stats.items()},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def fns_run(args, L, ctx, cfg, rank):
    """FNS++ pipeline of Sec. II.C on the GPU: truncation (Eq. 39-50, 41-44),
    ground state, and alpha at the config's frequencies, each timed."""
    import torch
    t0 = time.perf_counter()
    vk, occ = L.lrcc_fns_truncate(ctx, True, cfg["keep"])
    torch.cuda.synchronize()
    t_fns = time.perf_counter() - t0
    ef, et, de = L.lrcc_mp2_correction(ctx)
    t0 = time.perf_counter()
    E, itT, itL = L.lrcc_ccsd_ground(ctx)
    t_gs = time.perf_counter() - t0
    t0 = time.perf_counter()
    alpha, err = L.lrcc_solve(ctx, list(cfg["omegas"]), list(cfg["comps"]))
    t_sol = time.perf_counter() - t0
    n64, nmix = L.lrcc_solve_counts(ctx)
    nrhs = len(cfg["omegas"]) * len(cfg["comps"])
    if rank == 0:
        print(json.dumps({"metric": "FNS++ LR-CCSD pipeline", "workload": args.workload, "O": cfg["O"],
                          "V_full": cfg["V"], "V_kept": vk, "L": cfg["L"], "precision": args.prec,
                          "seconds": {"fns_truncate": t_fns, "ground": t_gs, "solve": t_sol},
                          "alpha_solves_per_s": nrhs / t_sol, "E_corr": [E.real, E.imag],
                          "dE_mp2": [de.real, de.imag], "iters_T": itT, "maps_L": itL,
                          "fp64_maps": n64, "mixed_maps": nmix, "occ_top": float(occ[0]),
                          "occ_kept_min": float(occ[vk - 1]), "occ_sum": float(occ.sum()),
                          "alpha_diag": [float(alpha[0, k, k].real) for k in range(len(cfg["comps"]))],
                          "alpha_iso": float(np.trace(alpha[0]).real / 3), "max_residual": float(err.max()),
                          "phase_ms": [round(x, 1) for x in L.lrcc_phase_times(ctx)]}), flush=True)


def ladder_only(args, L, ctx, O, V, Lx, R, prec, world, rank, local, pg):
    """The particle-particle ladder alone on R right-hand sides of the workload,
    on packed amplitudes (lrcc_ladder_packed_dev: only B_vv is read, so the
    largest virtual spaces fit).  <ab||ef> is cached when it fits in a third of
    the free memory, else assembled per call in slabs (counted in F_ladder)."""
    import torch
    dev = torch.device("cuda", local)
    po, pv = O * (O - 1) // 2, V * (V - 1) // 2
    g = torch.Generator(device=dev).manual_seed(7 + rank)
    xt = torch.randn(R * po, pv, dtype=torch.complex128, device=dev, generator=g)
    zt = torch.empty_like(xt)
    for _ in range(max(1, args.warmup)):
        L.lrcc_ladder_packed_dev(ctx, xt, prec=prec, out=zt)
    torch.cuda.synchronize()
    L.lrcc_profile(ctx, True)
    clocks = Clocks()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        ev[k][0].record()
        L.lrcc_ladder_packed_dev(ctx, xt, prec=prec, out=zt)
        ev[k][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    L.lrcc_profile(ctx, False)
    if args.profile_csv:
        L.lrcc_profile_dump(ctx, args.profile_csv)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    F = 8.0 * (R * po * pv * pv + pv * pv * Lx)
    stats = L.lrcc_kernel_stats(ctx)
    hbm, bf16, bf16s, src = load_peaks()
    # a ladder call runs for seconds at the large workloads: the sustained bf16 peak
    peak = {"bf16x3": bf16s / 3.0, "tf32": bf16s / 2.0}.get(args.prec)
    if rank == 0:
        line = {"metric": "ladder TFLOP/s (nominal F_ladder)", "value": world * F / (ms / 1e3) / 1e12,
                "unit": "TFLOP/s", "ms_per_step": ms, "steps": args.steps, "workload": args.workload,
                "O": O, "V": V, "L": Lx, "R": R, "ncol": R * po, "precision": args.prec, "clocks": clk,
                "F_ladder": F,
                "kernels": {k: {"count": v["count"], "ms": v["ms"] / args.steps,
                                "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9} for k, v in stats.items()}}
        if peak:
            line["frac_of_peak"] = line["value"] / peak
            line["peak"] = {"value": peak, "unit": "TFLOP/s",
                            "note": f"bf16 {src} sustained peak / {3 if args.prec == 'bf16x3' else 2} "
                                    "(useful complex flops, 8 per CMAC)"}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
