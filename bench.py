"""Benchmark: LR-CCSD residual throughput on one GB300 (or N replicas).

Workload (default): the dynamic-spectrum system O=28, V=600, L=1200 (seed 3),
one chunk of R right-hand sides of its 3 x 64 (component, frequency) spectrum,
linearised at the MP2 amplitudes (Eq. 39).  One step = the two residual maps
that every response iteration applies to a chunk: sigma = A X (Eq. 30) and the
transpose product A^T Y (left response, Eq. 32).
Metric: nominal complex flops per second,
    F_sigma = 8 [R (P_O P_V^2 + O^3 V^3) + P_V^2 L]   per map
(ladder contraction, ring, and the <ab||ef> assembly that each map needs once
at this size), counted once per map regardless of the contraction order or the
precision scheme.  The same line carries the FP64-class arm (the same step with
FP64-accurate products emulated on the tensor cores) and alpha(omega) solves/s
of the benchmark-size system (O=10, V=120), each alpha checked against the
FP64-class solve within 1e-6.

--impl reference times the CPU oracle (the plain complex128 PyTorch CPU
restatement, restricted to sampled residual rows) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
DEFAULT_RHS = {"c4": 4}


def nominal_flops(O, V, L, R, assembly=True):
    """F_sigma = 8 [R (P_O P_V^2 + O^3 V^3) + P_V^2 L]; the assembly term is left
    out when the <ab||ef> matrix is cached (it is then built once per context,
    not once per residual map)."""
    po, pv = O * (O - 1) // 2, V * (V - 1) // 2
    return 8.0 * (R * (po * pv * pv + O ** 3 * V ** 3) + (pv * pv * L if assembly else 0))


def assembly_per_call(O, V, L):
    """<ab||ef> does not fit in memory as a matrix (embedded: 12 bytes per
    complex element) when P_V^2 * 12 bytes exceeds a third of ~280 GB: then it
    is assembled in every map and its flops count."""
    pv = V * (V - 1) // 2
    return 12.0 * pv * pv > 0.33 * 280e9


def recorded_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary of this
    workload, or None when the kernel's source has changed since the counters
    were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", f"tc_gemm_traffic_{workload}.txt")
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
        if sha != kv.get("sha256_16"):
            return None
        return {"per_step": float(kv["bytes_per_step"]), "per_launch": float(kv["bytes_per_launch"]),
                "launches_per_step": int(kv["launches_per_step"])}
    return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return platform.processor() or platform.machine()


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


def workload_name(workload, cfg, R):
    nw = len(cfg["comps"]) * len(cfg["omegas"])
    return (f"{workload}: O={cfg['O']} V={cfg['V']} L={cfg['L']}, R={R} RHS per step (one chunk of the "
            f"{len(cfg['comps'])} comps x {len(cfg['omegas'])} omegas = {nw} RHS), MP2 linearisation, "
            f"sigma + A^T Y per step")


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------
# the CPU oracle on a bounded sample of the workload (reference arm and the
# cpu_baseline leg): the residual rows of a few occupied x virtual spinors
# ----------------------------------------------------------------------------

class OracleSample:
    """sigma rows and A^T lambda (lambda on the same rows) of the oracle at the
    workload's MP2 linearisation point, for a seeded row set; the setup (integral
    slices, MP2 amplitudes) happens once, outside the timed samples."""

    def __init__(self, cfg, n_occ=2, n_virt=3):
        import torch
        from oracle import ccsd, fns, sampled
        O, V = cfg["O"], cfg["V"]
        s = synth.make_system(O, V, cfg["L"], cfg["seed"], with_mu=False)
        rng = np.random.default_rng(4005)
        so = np.sort(rng.choice(O, min(n_occ, O), replace=False))
        sv = np.sort(rng.choice(V, min(n_virt, V), replace=False))
        self.model = sampled.RowModel(sampled.RowIntegrals(np.diag(s["eps"]).astype(np.complex128), O, s["B"],
                                                           so, sv))
        t2 = fns.mp2_doubles(s["eps"], s["B"], O)
        del s
        lay = self.model.lay
        self.t = lay.vec(torch.zeros(O, V, dtype=ccsd.CT), torch.as_tensor(t2))
        del t2
        a = synth.random_amplitudes(O, V, 1, seed=2000)
        self.x = lay.join(torch.as_tensor(a["t1"][0]), torch.as_tensor(a["t2u"][0]))
        sing, dbl = self.model.rows()
        self.n_rows = len(sing) + len(dbl)
        self.n_total = lay.n
        self.lam = torch.as_tensor(rng.standard_normal(self.n_rows) + 1j * rng.standard_normal(self.n_rows))
        self.desc = (f"residual rows of {len(so)} occupied x {len(sv)} virtual spinors ({self.n_rows} of "
                     f"{self.n_total} unique rows): sigma rows and A^T lambda with lambda on those rows, one RHS")

    def step(self):
        self.model.jvp(self.t, self.x)
        self.model.vjp(self.t, self.lam)

    def rate(self, seconds, O, V, L):
        """TFLOP/s by linear extrapolation in rows: the step's share of the
        nominal flops of sigma + A^T for one RHS is n_rows / n_total."""
        F = 2 * nominal_flops(O, V, L, 1, assembly=assembly_per_call(O, V, L))
        return F * (self.n_rows / self.n_total) / seconds / 1e12


def run_reference(args, world, rank):
    """CPU oracle on bounded samples of the same workload (all host cores)."""
    if rank != 0:
        return
    import torch
    cfg = synth.CONFIGS[args.workload]
    O, V, Lx = cfg["O"], cfg["V"], cfg["L"]
    R = args.rhs or DEFAULT_RHS.get(args.workload, len(cfg["comps"]) * len(cfg["omegas"]))
    smp = OracleSample(cfg)
    for _ in range(max(0, args.warmup)):
        smp.step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        smp.step()
        times.append(time.perf_counter() - t0)
    med = statistics.median(times)
    v = smp.rate(med, O, V, Lx)
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": "LR-CCSD residual TFLOP/s", "value": v, "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * med, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128 (f64, CPU)", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, cfg, R),
                       "flop_count": "2 x 8 [R (P_O P_V^2 + O^3 V^3) + P_V^2 L] per step of R RHS; each timed "
                                     "step here is a sample of sampled residual rows of one RHS, credited "
                                     "with its share of the rows (linear extrapolation in rows)"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": smp.desc,
                             "cpu": cpu_model(), "extrapolation": "linear in rows (labelled estimate)"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(cfg):
    """The oracle on sampled rows of the same workload: median of 3 samples on
    all host cores after one warm-up of both maps, and one sample on 1 core."""
    import torch
    O, V, Lx = cfg["O"], cfg["V"], cfg["L"]
    smp = OracleSample(cfg)
    smp.step()
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        smp.step()
        ts.append(time.perf_counter() - t0)
    med = statistics.median(ts)
    cores = torch.get_num_threads()
    torch.set_num_threads(1)
    t0 = time.perf_counter()
    smp.step()
    t1c = time.perf_counter() - t0
    torch.set_num_threads(cores)
    return {"value": smp.rate(med, O, V, Lx), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": smp.desc + f"; median of 3 samples ({med:.1f} s each)",
            "extrapolation": "linear in rows (labelled estimate)", "cpu": cpu_model(),
            "one_core": {"value": smp.rate(t1c, O, V, Lx), "seconds": t1c}}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def mp2_point(L, ctx, eps, O, V):
    """MP2 amplitudes (one Jacobi step from T = 0, Eq. 39) from the library's own
    residual at T = 0: t = -R(0) / D (singles vanish for the canonical reference)."""
    n1, n2 = O * V, O * O * V * V
    r0 = L.lrcc_residual(ctx, L.LRCC_RES_T, None, np.zeros((1, n1 + n2), np.complex128), prec=L.LRCC_MIXED_BF16X3)[0]
    eo, ev = eps[:O], eps[O:]
    t = np.zeros(n1 + n2, np.complex128)
    t[:n1] = -r0[:n1] / (ev[None, :] - eo[:, None]).reshape(-1)
    D2 = (ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None])
    t[n1:] = -r0[n1:] / D2.reshape(-1)
    return t


def timed_steps(L, ctx, x_dev, prec, steps, warmup, flush, pg=None, profile=False):
    import torch

    def step():
        L.lrcc_residual_dev(ctx, L.LRCC_RES_SIGMA, None, x_dev, prec=prec)
        L.lrcc_residual_dev(ctx, L.LRCC_RES_VJP, None, x_dev, prec=prec)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    if profile:
        L.lrcc_profile(ctx, True)
    launches0 = L.lrcc_kernel_launches(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.nvtx.range_push("timed")
    for k in range(steps):
        flush.zero_()                       # L2 flush between timed steps (256 MB > 129 MB L2)
        ev[k][0].record()
        step()
        ev[k][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if pg:
        pg.barrier()
    launches = (L.lrcc_kernel_launches(ctx) - launches0) // max(steps, 1)
    stats = None
    if profile:
        L.lrcc_profile(ctx, False)
        stats = L.lrcc_kernel_stats(ctx)
    return [a.elapsed_time(b) for a, b in ev], launches, stats


def alpha_solves(L, args, rank, world):
    """alpha(omega) solves/s on the benchmark-size system (O=10, V=120, 12 RHS):
    the mixed-precision solve timed, each alpha checked against the FP64-class
    (emulated FP64) solve of the same right-hand sides within 1e-6."""
    cfg = synth.CONFIGS["c2"]
    O, V = cfg["O"], cfg["V"]
    s = synth.make_system(O, V, cfg["L"], cfg["seed"])
    omegas = [w + 1e-3 * rank for w in cfg["omegas"]]   # weak scaling: each rank its own frequencies
    comps = list(cfg["comps"])
    out = {}
    alphas = {}
    for name in (args.prec, "fp64emu"):
        o = L.lrcc_default_options()
        o.prec = PREC_NAMES[name]
        o.solver = 1 if (args.solver == "subspace" and name == "fp64emu") else 0
        ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V, o)
        t0 = time.perf_counter()
        E, itT, itL = L.lrcc_ccsd_ground(ctx)
        tg = time.perf_counter() - t0
        t0 = time.perf_counter()
        alpha, err = L.lrcc_solve(ctx, omegas, comps)
        dt = time.perf_counter() - t0
        n64, nmix = L.lrcc_solve_counts(ctx)
        alphas[name] = alpha
        out[name] = {"seconds": dt, "ground_seconds": tg, "alpha_per_s": len(omegas) * len(comps) / dt,
                     "fp64_maps": n64, "mixed_maps": nmix, "max_residual": float(err.max()),
                     "E_corr": [E.real, E.imag], "iters_T": itT, "iters_L": itL}
        del ctx
    a, ref = alphas[args.prec], alphas["fp64emu"]
    R = len(omegas) * len(comps)
    # every (component, omega) pair: its diagonal alpha against the FP64-class value
    rel = np.array([abs(a[w, k, k] - ref[w, k, k]) / abs(ref[w, k, k])
                    for w in range(len(omegas)) for k in range(len(comps))])
    ok = int((rel <= 1e-6).sum())
    return {"value": world * ok / out[args.prec]["seconds"], "unit": "alpha(omega)/s (verified within 1e-6)",
            "workload": f"c2: O={O} V={V} L={cfg['L']}, {len(comps)} comps x {len(omegas)} omegas = {R} RHS, "
                        "ground state then X, F X, Y, alpha",
            "rhs": R, "verified": ok, "max_rel_err_vs_fp64emu": float(rel.max()),
            "rel_err_per_alpha": [float(x) for x in rel], "precision": args.prec,
            "mixed": out[args.prec], "fp64emu": out["fp64emu"],
            "fp64emu_value": world * R / out["fp64emu"]["seconds"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--rhs", type=int, default=0, help="right-hand sides per step (default: 4 at c4, all at c2)")
    ap.add_argument("--prec", default="bf16x3", choices=list(PREC_NAMES))
    ap.add_argument("--solver", default="diis", choices=["diis", "subspace"],
                    help="FP64-class solver of the alpha check: per right-hand-side DIIS or one shared subspace")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--fns", action="store_true",
                    help="FNS++ workload: truncate to the config's 'keep' virtuals, then ground state and alpha")
    ap.add_argument("--profile-csv", default=None,
                    help="write every timed GEMM launch (kernel, M, N, K, batch, ms, flops) to this CSV file")
    ap.add_argument("--ladder-only", action="store_true",
                    help="time only the particle-particle ladder (no ground state); used for kernel profiling")
    ap.add_argument("--solve", action="store_true",
                    help="one full lrcc_solve on the workload (ground state, then X, F X, Y and alpha for the "
                         "--solve-omegas and --solve-comps, --rhs right-hand sides per chunk), timed")
    ap.add_argument("--solve-omegas", default="0.0")
    ap.add_argument("--solve-comps", default="2")
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
    R = args.rhs or DEFAULT_RHS.get(args.workload, len(cfg["comps"]) * len(cfg["omegas"]))
    prec = PREC_NAMES[args.prec]
    s = synth.make_system(O, V, Lx, cfg["seed"])
    opt = L.lrcc_default_options()
    opt.prec = prec
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V, opt)
    if args.ladder_only:
        return ladder_only(args, L, ctx, O, V, Lx, R, prec, world, rank, local, pg)
    if args.solve:
        del ctx
        opt.rhs_chunk = args.rhs or 1
        ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V, opt)
        return solve_run(args, L, ctx, cfg, rank)
    if args.fns:
        opt.solver = 1 if args.solver == "subspace" else 0
        ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V, opt)
        return fns_run(args, L, ctx, cfg, rank)
    eps = s["eps"]
    del s
    # linearisation point: the MP2 amplitudes, primal evaluated once with
    # FP64-class products (outside timing)
    t0 = time.perf_counter()
    t_host = mp2_point(L, ctx, eps, O, V)
    L.lrcc_linearize(ctx, t_host, prec=L.LRCC_FP64_EMULATED)
    t_lin = time.perf_counter() - t0
    del t_host
    n_amp = O * V + O * O * V * V
    dev = torch.device("cuda", local)
    # R right-hand sides (seeded per rank); the residual maps project the
    # doubles block onto its antisymmetric part
    g = torch.Generator(device=dev).manual_seed(2000 + 17 * rank)
    x_dev = 0.05 * torch.randn(R, n_amp, dtype=torch.complex128, device=dev, generator=g)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = Clocks()
    clocks.start()
    ms, launches, stats = timed_steps(L, ctx, x_dev, prec, args.steps, max(3, args.warmup), flush, pg, profile=True)
    clk = clocks.stop()
    if args.profile_csv:
        L.lrcc_profile_dump(ctx, args.profile_csv)
    total = sum(ms)
    if pg:
        t = torch.tensor([total], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total = float(t.item())
    asm = assembly_per_call(O, V, Lx)
    F_step = 2 * nominal_flops(O, V, Lx, R, assembly=asm)
    value = world * F_step * args.steps / (total / 1e3) / 1e12

    # the FP64-class arm: the same step on the same inputs with FP64-accurate
    # products (emulated on the tensor cores); at this size one step runs for
    # a minute, so one timed step without warm-up (no caches are built at the
    # first call: <ab||ef> is assembled in every map)
    fp64_arm = None
    if not args.no_fp64_arm:
        ms64, l64, _ = timed_steps(L, ctx, x_dev, L.LRCC_FP64_EMULATED, 1, 0, flush, pg)
        t64 = sum(ms64)
        fp64_arm = {"precision": "fp64emu", "value": world * F_step / (t64 / 1e3) / 1e12, "unit": "TFLOP/s",
                    "ms_per_step": t64, "steps": 1, "warmup": 0,
                    "speedup_of_mixed": t64 / (total / args.steps)}

    # end to end through the host-buffer ABI: H2D of X, D2H of both results
    # (the device copy of the batch is released first: the host path stages
    # its own)
    x_host = x_dev.cpu().numpy()
    del x_dev
    torch.cuda.empty_cache()
    e2e_t = []
    for _ in range(2):
        t0 = time.perf_counter()
        L.lrcc_residual(ctx, L.LRCC_RES_SIGMA, None, x_host, prec=prec)
        L.lrcc_residual(ctx, L.LRCC_RES_VJP, None, x_host, prec=prec)
        e2e_t.append(time.perf_counter() - t0)
    e2e = F_step / min(e2e_t) / 1e12 * world
    h2d = 2 * x_host.nbytes
    d2h = 2 * x_host.nbytes
    del x_host, ctx
    torch.cuda.empty_cache()

    solves = None
    if not args.no_solve:
        torch.cuda.synchronize()
        solves = alpha_solves(L, args, rank, world)

    # roofline of the dominant kernel family in the timed region: the nominal
    # flops of the step are all contraction work, which that family executes
    hbm, bf16, bf16s, src = load_peaks()
    dom = max(stats.items(), key=lambda kv: kv[1]["ms"]) if stats else None
    roof = None
    if dom:
        name, st = dom
        t_k = st["ms"] / args.steps / 1e3                  # its time per step
        achieved = F_step / t_k / 1e12
        executed = st["flops"] / args.steps / t_k / 1e12
        if name == "gemm_tc_bf16x3":
            peak, unit, bound = bf16s / 3.0, "TFLOP/s", "tensor"     # 3 bf16 products per real product
            note = f"bf16 {src} sustained peak / 3 (bf16x3 split); complex flops counted 8 per CMAC"
        elif name == "gemm_tc_f64emu":
            peak, unit, bound = bf16s / 28.0, "TFLOP/s", "tensor"
            note = f"bf16 {src} sustained peak / 28 (7x6-bit slices, diagonals 0..6)"
        elif name == "gemm_tc_tf32":
            peak, unit, bound = bf16s / 2.0, "TFLOP/s", "tensor"     # tf32 dense = bf16 / 2 nominal
            note = f"bf16 {src} sustained peak x tf32/bf16 nominal ratio 1/2"
        else:
            peak, unit, bound = 1.25, "TFLOP/s", "alu"              # FP64 nominal (FMA pipes)
            note = "GB300 FP64 nominal 1.25 TFLOP/s"
        tr = recorded_traffic(name, args.workload)
        roof = {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": tr["per_step"] if tr else None,
                "traffic_unit": "DRAM bytes (read + write) per step of this kernel family, ncu capture in profiles/",
                "traffic_per_launch": tr["per_launch"] if tr else None,
                "launches": st["count"] // args.steps,
                "achieved_basis": "nominal F_step (2 F_sigma) / this family's device time per step",
                "executed_tflops": executed, "executed_frac": executed / peak,
                "share_of_step": st["ms"] / total, "peak_note": note}

    line = {
        "metric": "LR-CCSD residual TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[args.prec],
        "data": "synthetic",
        "config": {"workload": workload_name(args.workload, cfg, R),
                   "flops_per_step": F_step,
                   "flop_count": "2 x 8 [R (P_O P_V^2 + O^3 V^3) + P_V^2 L]" if asm else
                                 "2 x 8 R (P_O P_V^2 + O^3 V^3); <ab||ef> cached, not counted",
                   "l2": "flushed (256 MB write) between timed steps; inputs larger than L2",
                   "linearisation_seconds": t_lin,
                   "parallelism": f"replicas x{world} (RHS sharding, no collective)"},
        "e2e": {"value": e2e, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clk, "roofline": roof, "fp64_class_arm": fp64_arm,
        "alpha_solves": solves,
        "kernels": {k: {"count": v["count"] // args.steps, "ms_per_step": v["ms"] / args.steps}
                    for k, v in (stats or {}).items()},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def solve_run(args, L, ctx, cfg, rank):
    """Ground state (T, Lambda) and the linear-response solves of Eq. 29-35 on the
    workload's system through the C ABI, each phase timed."""
    omegas = [float(x) for x in args.solve_omegas.split(",")]
    comps = [int(x) for x in args.solve_comps.split(",")]
    t0 = time.perf_counter()
    E, itT, itL = L.lrcc_ccsd_ground(ctx)
    t_gs = time.perf_counter() - t0
    n64g, nmixg = L.lrcc_solve_counts(ctx)
    t0 = time.perf_counter()
    alpha, err = L.lrcc_solve(ctx, omegas, comps)
    t_sol = time.perf_counter() - t0
    n64, nmix = L.lrcc_solve_counts(ctx)
    if rank == 0:
        print(json.dumps({"metric": "LR-CCSD alpha(omega) through lrcc_solve", "workload": args.workload,
                          "O": cfg["O"], "V": cfg["V"], "L": cfg["L"], "precision": args.prec,
                          "omegas": omegas, "comps": comps, "rhs_chunk": args.rhs or 1,
                          "seconds": {"ground": t_gs, "solve": t_sol},
                          "alpha_solves_per_s": len(omegas) * len(comps) / t_sol,
                          "E_corr": [E.real, E.imag], "iters_T": itT, "maps_L": itL,
                          "fp64_class_maps": n64, "mixed_maps": nmix,
                          "alpha": [[[[float(alpha[w, a, b].real), float(alpha[w, a, b].imag)]
                                      for b in range(len(comps))] for a in range(len(comps))]
                                    for w in range(len(omegas))],
                          "max_residual": float(err.max()),
                          "phase_ms": [round(x, 1) for x in L.lrcc_phase_times(ctx)]}), flush=True)


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
