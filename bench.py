"""Benchmark: shift-solves/s of the batched shifted m-Hessenberg solver on GB300.

One step = the whole path over one synthetic system: the FP64 controller-
Hessenberg reduction of (A, B, C) followed by the solve of every shift,
G(sigma_j) = C (A - sigma_j I)^{-1} B.  The workload is n = 5000, m = p = 16,
2000 shifts on the 50 x 40 grid over [-4, 0] x [-2, 2] (A = -2I + G/sqrt(n)).
value = shifts processed by all ranks / max-over-ranks time of K steps of the
headline precision (default: the certified mixed path); the FP64 and
double-float steps are timed beside it for the comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64|dfloat]
    python bench.py --impl reference ...   # the CPU oracle arm

Under torchrun each rank solves its own copy of the workload (weak scaling;
shifts are independent, there is no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "shift-solves/s at n=5000,m=16 (mixed vs FP64, resid<=1e-12); p50/p99 latency"
# DRAM bytes of one reduce_blocked_kernel launch at n = 5000, m = p = 16 (ncu), or None
REDUCE_TRAFFIC_N5000_M16 = 130381078528 + 90573036032
# dram__bytes_read.sum + dram__bytes_write.sum of all tcs_update_kernel launches of one
# 304-shift sweep of this workload, per shift (profiles/tcs_sweep_n5000_m16_304shifts.md);
# the window state it streams is per shift, so traffic scales with the shifts
TCS_UPDATE_TRAFFIC_PER_SHIFT = (17579877120 + 18607825408) / 304.0
UNIT = "shift-solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "dfloat", "split"], default="mixed",
                    help="headline precision (value, e2e, roofline); the others are timed beside it "
                         "(--profile-solve: the precision of the profiled solve)")
    ap.add_argument("--first", choices=["tensor", "dfloat", "c64"], default="tensor",
                    help="first solve of the mixed path")
    ap.add_argument("--reduce", choices=["auto", "fp64", "tensor"], default="auto",
                    help="arithmetic of the reduction's bulk products; auto: FP64 for the fp64 "
                         "step, the tensor-core form for the others")
    ap.add_argument("--side-steps", type=int, default=5,
                    help="timed steps of the comparison precisions")
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-shifts", type=int, default=16)
    ap.add_argument("--shifts", type=int, default=0,
                    help="solve only this many evenly spread grid shifts (profiling); 0 = all")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batching and serving measurements")
    ap.add_argument("--serving-scale", type=float, default=1.0)
    ap.add_argument("--serving-requests", type=int, default=400)
    ap.add_argument("--serving-budget-gb", type=float, default=16.0)
    ap.add_argument("--profile-reduce", type=int, default=0,
                    help="profiling case: one reduction of an n x n system (m = p = --profile-m)")
    ap.add_argument("--profile-m", type=int, default=16)
    ap.add_argument("--profile-resid", action="store_true",
                    help="one tensor-core backward-error pass of the workload (for ncu)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="profiling case: one solve on a handle restored from an m-Hessenberg "
                         "stand-in (H = triu(A, -m), R = triu(B), Ct = C), no reduction")
    return ap.parse_args()


def reduce_arith(args, precision):
    if args.reduce != "auto":
        return args.reduce
    return "fp64" if precision == "fp64" else "tensor"


def workload_config(sysr, sig, nb, precision, arith="fp64"):
    red = ("FP64 reduction" if arith == "fp64" else
           "reduction with tensor-core digit products (FP64 accuracy)")
    return {
        "workload": "precision grid: n=%d, m=p=%d, %d shifts on the 50x40 grid over [-4,0]x[-2,2], "
                    "A=-2I+G/sqrt(n)" % (sysr.n, sysr.m, len(sig)),
        "n": sysr.n, "m": sysr.m, "p": sysr.p, "shifts": int(len(sig)),
        "output": "G(sigma)=C X, complex128, p x (s*m)",
        "step": "%s + %s solve of all shifts (certified: backward error <= 1e-12)"
                % (red, precision), "reduce": arith,
        "precision": precision, "nb": nb or (128 if sysr.n >= 1024 else 64),
        "l2": "inputs larger than L2 (A and H are 200 MB each; every step re-reads A)",
    }


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": float(max(power))}


# ----------------------------------------------------------------------------
# the oracle (CPU) arm
# ----------------------------------------------------------------------------
def oracle_sample(sig, k):
    """k grid shifts: three quarters inside the spectral disc |sigma + 2| < 1 (where the
    condition numbers are large), the rest outside, evenly spread over each set."""
    inside = np.where(np.abs(sig + 2.0) < 1.0)[0]
    outside = np.where(np.abs(sig + 2.0) >= 1.0)[0]
    ki = (3 * k) // 4
    return np.concatenate([inside[np.linspace(0, len(inside) - 1, ki).astype(int)],
                           outside[np.linspace(0, len(outside) - 1, k - ki).astype(int)]])


def cpu_baseline_leg(ssv, sysr, sig, dev, args):
    """The oracle as it stands on the host cores: its reduction of the full system
    plus tier-2 reduced GEPP on a sample of grid shifts (one call, parallel over the
    shifts), extrapolated to all shifts.  On the same sample, the per-shift relative
    error of the GPU's G (mixed and FP64 paths) against the oracle's G, with the
    oracle's condition estimate kappa_1 beside it."""
    import torch

    import oracle

    oracle._load()
    cores = os.cpu_count()
    pick = oracle_sample(sig, max(4, args.cpu_shifts))
    t0 = time.perf_counter()
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    t_red = time.perf_counter() - t0
    t0 = time.perf_counter()
    Go, sto, _ = oracle.reduced_solve(Ho, Ro, Co, sig[pick], want="g")
    t_call = time.perf_counter() - t0
    per_shift = t_call / len(pick)
    value = len(sig) / (t_red + per_shift * len(sig))
    _, _, k1 = oracle.reduced_solve(Ho, Ro, Co, sig[pick], want="g", cond=True)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).t().contiguous().t().to(dev)  # noqa
    h = ssv.reduce(to(sysr.A), to(sysr.B), to(sysr.C))
    sd = torch.from_numpy(sig[pick].astype(np.complex128)).to(dev)
    errs = {}
    for prec in ("mixed", "fp64"):
        out, st, resid = h.solve(sd, mode="g", precision=prec, want_resid=True)
        G = out.cpu().numpy()
        m = sysr.m
        errs[prec] = [float(np.linalg.norm(G[:, j * m:(j + 1) * m] - Go[j]) / np.linalg.norm(Go[j]))
                      for j in range(len(pick))]
        errs[prec + "_eta"] = [float(x) for x in resid.cpu().numpy()]
    h.close()
    gate = k1 <= 1e6
    r3 = lambda xs: [float("%.3g" % x) for x in xs]  # noqa: E731
    return {
        "value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": "oracle reduction of the full n=5000 system (%.1f s) + tier-2 reduced GEPP on "
                  "%d grid shifts (%d inside the spectral disc) in one call, %.3f s/shift, "
                  "extrapolated to %d shifts" % (t_red, len(pick), (3 * len(pick)) // 4,
                                                 per_shift, len(sig)),
        "per_shift_error": {
            "reference": "oracle: own reduction + tier-2 reduced GEPP, G = Ct Xhat; "
                         "rel_err = ||G - G_oracle||_F / ||G_oracle||_F",
            "sigma_re": r3(sig[pick].real), "sigma_im": r3(sig[pick].imag), "kappa1": r3(k1),
            "rel_err_mixed": r3(errs["mixed"]), "rel_err_fp64": r3(errs["fp64"]),
            "backward_error_mixed": r3(errs["mixed_eta"]),
            "max_rel_err_mixed_kappa_le_1e6": float(max(np.array(errs["mixed"])[gate], default=0.0)),
            "max_rel_err_fp64_kappa_le_1e6": float(max(np.array(errs["fp64"])[gate], default=0.0)),
            "oracle_status_nonzero": int((sto != 0).sum()),
        },
    }


def run_reference(args):
    """The oracle arm: the plain CPU oracle on the host cores.  One step = one
    tier-2 call on os.cpu_count() grid shifts (the call is parallel over shifts,
    one per core) plus that many shifts' share of the oracle reduction, which is
    timed once before the steps; value = shifts per second of that step, i.e.
    2000 / (t_reduce + 2000 t_call / shifts_per_call)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sysr, sig = W.workload_precision()
    import oracle

    oracle._load()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    H, R, Ct, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    t_red = time.perf_counter() - t0
    per_step = cores
    idx_all = np.unique(np.linspace(0, len(sig) - 1, per_step * (args.steps + args.warmup)).astype(int))
    times = []
    for k in range(args.warmup + args.steps):
        idx = idx_all[(k * per_step) % len(idx_all):][:per_step]
        if len(idx) < per_step:
            idx = idx_all[:per_step]
        t0 = time.perf_counter()
        oracle.reduced_solve(H, R, Ct, sig[idx], want="g")
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t_call = float(np.mean(times))
    step_s = t_call + t_red * per_step / len(sig)
    value = per_step / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(sysr, sig, 0, args.precision, reduce_arith(args, args.precision)),
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                         "sample": "per step: oracle tier-2 reduced GEPP on %d grid shifts in one "
                                   "call (parallel over shifts, %.3f s) + those shifts' share of "
                                   "the oracle reduction of the full n=5000 system (%.1f s, timed "
                                   "once)" % (per_step, t_call, t_red)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# multi-rank aggregation (weak scaling: every rank solves its own copy)
# ----------------------------------------------------------------------------
def combine_ranks(world, shifts_per_rank, steps, local_ms, reduce_max):
    """Whole-job throughput: shifts of all ranks over the slowest rank's time."""
    total_ms = reduce_max(local_ms)
    return world * shifts_per_rank * steps / (total_ms * 1e-3), total_ms


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
def serving_measurement(ssv, dev, args):
    """The serving workload: 8 preloaded reduced systems (n = 1000 .. 10000,
    m = (1, 4, 16)[i % 3], p = m), requests of 1..256 imaginary-axis shifts,
    solved with the certified mixed path.  Saturated throughput first (every
    request at t = 0), then Poisson arrivals at 0.5 / 0.8 / 0.95 of it, each
    with --serving-requests requests; p50 / p99 latency per load."""
    import torch

    from paper_1708_06290_gb300.serve import Server, make_requests

    systems = W.workload_serving_systems(scale=args.serving_scale)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).t().contiguous().t().to(dev)  # noqa
    handles = [ssv.reduce(to(sy.A), to(sy.B), to(sy.C)) for sy in systems]
    torch.cuda.synchronize()
    budget = int(args.serving_budget_gb * (1 << 30))
    nreq = args.serving_requests
    prec = "mixed"
    warm = make_requests(W.serving_requests(16, 100.0, seed=900))
    Server(handles, slots=4, mem_budget=budget, precision=prec).run(warm, realtime=False)
    sat = Server(handles, slots=4, mem_budget=budget, precision=prec).run(
        make_requests(W.serving_requests(nreq, 1.0, seed=901)), realtime=False)
    req_rate = sat["requests"] / sat["wall_s"]
    loads = {}
    for f in (0.5, 0.8, 0.95):
        st = Server(handles, slots=4, mem_budget=budget, precision=prec).run(
            make_requests(W.serving_requests(nreq, f * req_rate, seed=902 + int(100 * f))),
            realtime=True)
        loads["%.2f" % f] = {"p50_ms": round(st["p50_ms"], 2), "p99_ms": round(st["p99_ms"], 2),
                             "shift_solves_per_s": round(st["shift_solves_per_s"], 1),
                             "requests": st["requests"], "overlap": st["max_inflight_batches"]}
    for h in handles:
        h.close()
    return {"precision": prec, "requests_per_load": nreq,
            "saturated_shift_solves_per_s": round(sat["shift_solves_per_s"], 1),
            "saturated_requests_per_s": round(req_rate, 2), "poisson": loads}


def batching_measurement(ssv, dev, args):
    """The batching workload: 64 systems, n ~ U{200..3000}, m in {1,2,4,8},
    16..512 shifts each; n_b autotuned per system, then one batch plan per
    precision (FP64, double-float) captured in a CUDA graph and replayed
    (median of 3 replays); the mixed path through ssv_solve_many; reductions
    and tuning untimed."""
    import torch

    work = W.workload_batching()
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).t().contiguous().t().to(dev)  # noqa
    handles = [ssv.reduce(to(sy.A), to(sy.B), to(sy.C)) for sy, _ in work]
    shifts = [torch.from_numpy(sig.astype(np.complex128)).to(dev) for _, sig in work]
    total = sum(int(x.numel()) for x in shifts)
    res = {"systems": len(work), "shifts": total, "graph_replay": True}
    stream = torch.cuda.Stream()
    for prec in ("fp64", "dfloat"):
        tuned = [ssv.autotune(h, x, mode="g", precision=prec)[0] for h, x in zip(handles, shifts)]
        plan = ssv.BatchPlan(handles, shifts, mode="g", precision=prec)
        plan.run(stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            plan.run(stream)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        bad = int(sum(int((st != 0).sum()) for st in plan.statuses))
        res[prec] = {"ms": round(ms, 3), "shift_solves_per_s": round(total / (ms * 1e-3), 1),
                     "nb_tuned": sorted(set(tuned)), "nonzero_status": bad}
        plan.close()
        del g
    # the mixed path (certified per shift): ssv_solve_many runs the systems' mixed solves
    # back to back; the mixed path takes its scratch per call, so it is timed directly
    # (median of 3), not replayed from a graph.  An extra measurement: a failure is
    # reported on the line, not raised.
    try:
        ssv.solve_many(handles, shifts, mode="g", precision="mixed", stream=stream)
        torch.cuda.synchronize()
        ts, bad = [], 0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, sts = ssv.solve_many(handles, shifts, mode="g", precision="mixed", stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            bad = int(sum(int((x != 0).sum()) for x in sts))
        ms = float(np.median(ts))
        res["mixed"] = {"ms": round(ms, 3), "shift_solves_per_s": round(total / (ms * 1e-3), 1),
                        "graph_replay": False, "nonzero_status": bad}
    except Exception as exc:  # noqa: BLE001
        res["mixed"] = {"error": str(exc)[:200]}
    for h in handles:
        h.close()
    return res


def bf16_peak_sustained():
    """The sustained BF16 figure of MEASURED_PEAKS.json (the kernels below are timed inside
    a long step), else the recipe's fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback sustained BF16 1.7 PFLOP/s (of fallback)"


def tensor_residual_roofline(n, m, s, mixed):
    """BF16 tensor work of one certification pass of the mixed path: per shift and
    128-row block I, 36 digit-slice products of 128 x 32 x (K from column I*128-m)."""
    npad = (n + 127) // 128 * 128
    k_total = sum(npad - (max(0, i0 - m) // 32) * 32 for i0 in range(0, npad, 128))
    flops = 2.0 * 36 * 128 * 32 * k_total * s
    ms = mixed["phase_ms_per_step"].get("mixed_residual", float("nan"))
    peak, src = bf16_peak_sustained()
    ach = flops / (ms * 1e-3) / 1e12
    return {"kernel": "tc_residual2_kernel (two shifts per item, + digit split of Xhat)", "bound": "tensor",
            "unit": "TFLOP/s", "achieved": ach, "peak": peak, "frac": ach / peak,
            "peak_source": src,
            "flops_per_pass": flops, "pass_ms": ms,
            "flops_definition": "executed BF16 products: 36 slice pairs x 2 x 128 x 32 x K per "
                                "(shift, 128-row block); K = npad - 32 floor((128 I - m) / 32)"}


def tcs_update_flops(n, m, s):
    """Executed BF16 flops of all tcs_update_kernel launches of one tensor-core sweep (the
    loop of solve_tc): per item (128 rows above the block x one group of S = 64 / 2m shifts)
    ceil(nbe / 32) stages of 35 digit pairs x 2 K-halves of 128 x 64 x 16, then per shift 28
    pairs x 2 K-halves of 128 x 2m x 16 (Z2 P2).  Valid for 2m dividing 64."""
    cs = 2 * m
    if 64 % cs:
        return None, 0
    S = 64 // cs
    G = -(-s // S)
    nbe_first = (n - m) % 128 or 128
    k, step, flops, launches = n, 0, 0.0, 0
    while k > m:
        nbe = nbe_first if step == 0 else 128
        step += 1
        hrows = k - nbe
        if hrows > 0:
            items = -(-hrows // 128) * G
            per_item = -(-nbe // 32) * 70 * 2.0 * 128 * 64 * 16 + S * 56 * 2.0 * 128 * cs * 16
            flops += items * per_item
            launches += 1
        k -= nbe
    return flops, launches


def profile_resid(args):
    """The tensor-core backward error of the workload's first solve: split of H, split
    of Xhat and tc_residual_kernel, after one double-float solve in mode xhat."""
    import torch

    from paper_1708_06290_gb300 import ssv

    sysr, sig = W.workload_precision()
    if args.shifts:
        sig = sig[np.unique(np.linspace(0, len(sig) - 1, args.shifts).astype(int))]
    m = sysr.m
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).t().contiguous().t().cuda()  # noqa
    h = ssv.load_reduced(dev(np.triu(sysr.A, -m)), dev(np.triu(sysr.B)), dev(sysr.C))
    sd = torch.from_numpy(sig.astype(np.complex128)).cuda()
    X, st, _ = h.solve(sd, mode="xhat", precision="dfloat")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    eta = h.backward_error(sd, X, method="tensor")
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile": "resid", "n": sysr.n, "m": m, "shifts": int(len(sig)),
                      "ms": e0.elapsed_time(e1), "max_eta": float(eta.max().item()),
                      "nonzero_status": int((st != 0).sum())}))
    h.close()
    return 0


def profile_solve(args):
    """One solve of the workload's shifts on a restored stand-in handle: the solve
    kernels run after only the handful of launches that restore the handle."""
    import torch

    from paper_1708_06290_gb300 import ssv

    sysr, sig = W.workload_precision()
    if args.shifts:
        sig = sig[np.unique(np.linspace(0, len(sig) - 1, args.shifts).astype(int))]
    m = sysr.m
    Hs = np.triu(sysr.A, -m)
    Rs = np.triu(sysr.B)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).t().contiguous().t().cuda()  # noqa
    h = ssv.load_reduced(dev(Hs), dev(Rs), dev(sysr.C))
    sd = torch.from_numpy(sig.astype(np.complex128)).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out, st, _ = h.solve(sd, mode="g", precision=args.precision, nb=args.nb, first=args.first)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile": "solve", "precision": args.precision, "first": args.first,
                      "n": sysr.n, "m": m,
                      "shifts": int(len(sig)), "ms": e0.elapsed_time(e1),
                      "nonzero_status": int((st != 0).sum())}))
    h.close()
    return 0


def profile_reduce(args):
    """One controller-Hessenberg reduction (a single persistent kernel launch)."""
    import torch

    from paper_1708_06290_gb300 import ssv

    n = args.profile_reduce
    sysr = W.random_system(n, args.profile_m, args.profile_m, seed=77)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).t().contiguous().t().cuda()  # noqa
    A, B, C = dev(sysr.A), dev(sysr.B), dev(sysr.C)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    arith = "fp64" if args.reduce == "auto" else args.reduce
    h = ssv.reduce(A, B, C, arith=arith)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "reduce", "arith": arith, "n": n, "m": args.profile_m,
                      "s": time.perf_counter() - t0}))
    h.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_reduce:
        return profile_reduce(args)
    if args.profile_solve:
        return profile_solve(args)
    if args.profile_resid:
        return profile_resid(args)

    import torch
    import torch.distributed as dist

    from paper_1708_06290_gb300 import ssv

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world > 1:
            tt = torch.tensor([x], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            return float(tt.item())
        return x

    ssv.load()
    sysr, sig = W.workload_precision()
    if args.shifts:
        sig = sig[np.unique(np.linspace(0, len(sig) - 1, args.shifts).astype(int))]
    n, m, p, s = sysr.n, sysr.m, sysr.p, len(sig)

    def to_dev(a, dtype=torch.float64):
        t = torch.from_numpy(np.ascontiguousarray(a))
        if t.dim() == 2:
            t = t.t().contiguous().t()
        return t.to(dev, dtype)

    A_d, B_d, C_d = to_dev(sysr.A), to_dev(sysr.B), to_dev(sysr.C)
    sig_d = torch.from_numpy(sig.astype(np.complex128)).to(dev)
    out = torch.empty((s * m, p), dtype=torch.complex128, device=dev).t()
    status = torch.empty(s, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(precision):
        h = ssv.reduce(A_d, B_d, C_d, arith=reduce_arith(args, precision))
        h.solve(sig_d, mode="g", precision=precision, nb=args.nb, out=out, status=status)
        return h

    def timed(precision, steps, warmup):
        """W warm-up steps, then K steps bracketed by barrier + sync; phase spans
        from the library tracer (CUDA events on this stream)."""
        h = step(precision)
        _, st_chk, resid = h.solve(sig_d, mode="g", precision=precision, nb=args.nb,
                                   want_resid=True)
        torch.cuda.synchronize()
        gate = {"max_backward_error": float(resid.max()), "nonzero_status": int((st_chk != 0).sum())}
        h.close()
        for _ in range(warmup):
            step(precision).close()
        torch.cuda.synchronize()
        ssv.refine_counts(reset=True)
        ssv.trace(True)
        launches0 = ssv.kernel_launches()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        handles = []
        for _ in range(steps):
            handles.append(step(precision))
            if len(handles) > 1:
                handles.pop(0).close()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        for hh in handles:
            hh.close()
        launches = ssv.kernel_launches() - launches0
        phases = ssv.trace_read()
        ssv.trace(False)
        corr, resol = ssv.refine_counts(reset=True)
        value, total_ms = combine_ranks(world, s, steps, e0.elapsed_time(e1), max_over_ranks)
        phase_ms = {k: round(v[0] / steps, 3) for k, v in phases.items()}
        phase_calls = {k: int(v[1]) for k, v in phases.items()}
        return {"value": value, "ms_per_step": total_ms / steps, "steps": steps,
                "phase_ms_per_step": phase_ms, "phase_calls": phase_calls, "gpu_launches": int(launches),
                "corrections_per_step": corr / steps, "fp64_resolves_per_step": resol / steps,
                **gate}

    fp64_peak = ssv.peak_probe("fp64")
    fp32_peak = ssv.peak_probe("fp32")
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    headp = args.precision
    res = {headp: timed(headp, args.steps, args.warmup)}
    for prec in ("fp64", "mixed", "dfloat"):
        if prec != headp:
            res[prec] = timed(prec, max(1, min(args.side_steps, args.steps)), min(args.warmup, 3))
    clocks = clk.stop()
    head = res[headp]

    # ---- end to end through the public API with host buffers (headline precision)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    A_h = pin(sysr.A.T.copy())
    B_h = pin(sysr.B.T.copy())
    C_h = pin(sysr.C.T.copy())
    sig_h = pin(sig.astype(np.complex128))
    G_h = torch.empty((s * m, p), dtype=torch.complex128).pin_memory()
    st_h = torch.empty(s, dtype=torch.int32).pin_memory()
    A_e = torch.empty((n, n), dtype=torch.float64, device=dev)
    B_e = torch.empty((m, n), dtype=torch.float64, device=dev)
    C_e = torch.empty((n, p), dtype=torch.float64, device=dev)
    sig_e = torch.empty(s, dtype=torch.complex128, device=dev)
    h2d = (A_h.numel() + B_h.numel() + C_h.numel()) * 8 + sig_h.numel() * 16
    d2h = G_h.numel() * 16 + st_h.numel() * 4

    def e2e_step():
        A_e.copy_(A_h, non_blocking=True)
        B_e.copy_(B_h, non_blocking=True)
        C_e.copy_(C_h, non_blocking=True)
        sig_e.copy_(sig_h, non_blocking=True)
        hh = ssv.reduce(A_e.t(), B_e.t(), C_e.t(), arith=reduce_arith(args, headp))
        o, st2, _ = hh.solve(sig_e, mode="g", precision=headp, nb=args.nb)
        G_h.copy_(o.t(), non_blocking=True)
        st_h.copy_(st2, non_blocking=True)
        torch.cuda.synchronize()
        hh.close()

    e2e_value = None
    if args.e2e_steps > 0:
        e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        e2e_value = world * s * args.e2e_steps / e2e_s

    # ---- rooflines: the first-solve sweep of the mixed step (its largest phase) and
    # the FP64 sweep of the FP64 step
    floor_macs = n * n * m + 2.0 * n * m * p      # n_b-independent multiply-adds per shift
    fp64_ms = res["fp64"]["phase_ms_per_step"].get("solve_fp64", float("nan"))
    fp64_ach = 2.0 * floor_macs * s / (fp64_ms * 1e-3) / 1e12
    roof_fp64 = {
        "kernel": "solve_fp64_kernel", "bound": "alu", "unit": "TFLOP/s",
        "achieved": fp64_ach, "peak": fp64_peak, "frac": fp64_ach / fp64_peak,
        "peak_source": "FP64 DFMA probe measured in this run (nominal GB300 FP64 1.25 TFLOP/s)",
        "launch_ms": fp64_ms,
        "flops_definition": "2 n^2 m + 4 n m p per shift (trailing update Z1 P1 + Ct rows)",
        # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 152 shifts of
        # this workload (profiles/solve_fp64_kernel_n5000_m16_152shifts.md), scaled by shifts:
        # each shift streams its own Z2 state
        "traffic": (3.002227e9 + 3.462814e9) * s / 152.0 if args.nb in (0, 128) else None,
    }
    sweep0_ms = res["mixed"]["phase_ms_per_step"].get("mixed_sweep0", float("nan"))
    # the double-float equivalent of the first solve: each double-float multiply-add issues
    # 12 FP32-pipe instructions; the FFMA probe's TFLOP/s / 2 is the pipe's instruction rate
    instr = 12.0 * floor_macs * s
    ach_ti = instr / (sweep0_ms * 1e-3) / 1e12
    peak_ti = fp32_peak / 2.0
    roof_first = {
        "kernel": "tcs_panel_kernel + tcs_update_kernel<true> (tensor-core sweep, first solve of "
                  "the mixed path; %d launches each)" % (len(range(0, n - m, 128)) or 1),
        "bound": "alu", "unit": "T FP32-instr/s (double-float equivalent)", "achieved": ach_ti,
        "peak": peak_ti, "frac": ach_ti / peak_ti,
        "peak_source": "FFMA probe measured in this run / 2 (instructions/s; nominal 128 lanes x "
                       "152 SMs x 2.07 GHz = 40.3 T/s)",
        "launch_ms": sweep0_ms,
        "definition": "n_b-independent floor n^2 m + 2 n m p real multiply-adds per shift counted "
                      "at the 12 FP32 instructions a double-float multiply-add takes; the sweep "
                      "runs the Z1 P1 and Z2 P2 products as exact BF16 digit products on the "
                      "tensor cores instead, so this is the rate a double-float sweep would need",
        "traffic": None,
    }
    # the reduction of the mixed step (tensor-core form unless --reduce fp64): FP64-equivalent
    # rate against the DFMA peak, so a fraction above 1 is a reduction faster than the FP64
    # pipe could run it
    red_phases = res["mixed"]["phase_ms_per_step"]
    red_tc = "reduce_tc" in red_phases
    red_ms = red_phases.get("reduce_tc", red_phases.get("reduce", float("nan")))
    red_flops = 10.0 / 3.0 * n ** 3 - 4.5 * n * n * m
    red_ach = red_flops / (red_ms * 1e-3) / 1e12
    roof_reduce = {
        "kernel": ("tensor-core reduction (panel_kernel, tc_gemm_kernel<16,9> / <32,9> / <64,8>, "
                   "digit splits; about 1400 launches)" if red_tc else
                   "reduce_blocked_kernel (FP64 controller-Hessenberg reduction, one launch)"),
        "bound": "alu", "unit": "TFLOP/s (FP64-equivalent)", "achieved": red_ach, "peak": fp64_peak,
        "frac": red_ach / fp64_peak,
        "peak_source": "FP64 DFMA probe measured in this run (nominal GB300 FP64 1.25 TFLOP/s)",
        "launch_ms": red_ms,
        "flops_definition": "10/3 n^3 - 9/2 n^2 m (the blocking-independent terms of the "
                            "paper's reduction count)",
        # ncu dram__bytes_read.sum + dram__bytes_write.sum of the FP64 reduction launch at
        # n = 5000, m = p = 16 (profiles/reduce_blocked_kernel_n5000_m16.md)
        "traffic": (REDUCE_TRAFFIC_N5000_M16 if (n, m, p) == (5000, 16, 16) and not red_tc else None),
    }
    # the largest kernel of the mixed step by time: the tensor-core sweep's update, timed
    # per launch by the library's tracer spans (CUDA events on the solve's stream)
    upd_tot = res["mixed"]["phase_ms_per_step"].get("tcs_update", float("nan")) * res["mixed"]["steps"]
    upd_calls = res["mixed"]["phase_calls"].get("tcs_update", 0)
    upd_flops, upd_launches = tcs_update_flops(n, m, s)
    bf16_peak, bf16_src = bf16_peak_sustained()
    roof_update = None
    if upd_flops and upd_calls:
        upd_ms = upd_tot / upd_calls
        ach_u = upd_flops / upd_launches / (upd_ms * 1e-3) / 1e12
        roof_update = {
            "kernel": "tcs_update_kernel<true> (tensor-core sweep trailing update, %d launches "
                      "per solve)" % upd_launches,
            "bound": "tensor", "unit": "TFLOP/s", "achieved": ach_u, "peak": bf16_peak,
            "frac": ach_u / bf16_peak, "peak_source": bf16_src, "launch_ms": upd_ms,
            "flops_definition": "executed BF16 digit products per launch, averaged over the "
                                "solve's launches (bench.py tcs_update_flops)",
            "traffic": (TCS_UPDATE_TRAFFIC_PER_SHIFT * s / upd_launches
                        if TCS_UPDATE_TRAFFIC_PER_SHIFT and (n, m) == (5000, 16) else None),
        }
    roofline = (roof_update if headp in ("mixed", "split") and roof_update else
                (roof_reduce if headp != "fp64" else roof_fp64))
    mx = res["mixed"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32-pair+bf16-tc+f64", "fp64": "f64", "dfloat": "f32-pair"}[headp],
        "data": "synthetic",
        "config": workload_config(sysr, sig, args.nb, headp, reduce_arith(args, headp)),
        "mixed_value": mx["value"], "fp64_value": res["fp64"]["value"],
        "dfloat_value": res["dfloat"]["value"],
        "mixed_speedup_vs_fp64": mx["value"] / res["fp64"]["value"],
        "mixed_max_backward_error": mx["max_backward_error"],
        "mixed_nonzero_status": mx["nonzero_status"],
        "mixed_corrections_per_step": mx["corrections_per_step"],
        "mixed_fp64_resolves_per_step": mx["fp64_resolves_per_step"],
        "fp64_max_backward_error": res["fp64"]["max_backward_error"],
        "roofline": roofline,
        "roofline_reduction": roof_reduce,
        "roofline_first_solve": roof_first,
        "roofline_fp64_sweep": roof_fp64,
        "phase_ms": {k: res[k]["phase_ms_per_step"] for k in ("mixed", "fp64", "dfloat")},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": head["gpu_launches"],
        "fp32_ffma_peak_tflops": fp32_peak,
        "tensor_residual_roofline": tensor_residual_roofline(n, m, s, mx),
    }
    if not args.no_extras and world == 1:
        line["batching"] = batching_measurement(ssv, dev, args)
        line["serving"] = serving_measurement(ssv, dev, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(ssv, sysr, sig, dev, args)
    # the comparison once more, last on the line, so a truncated tail still has it
    line["summary"] = ("%s step %.1f shift-solves/s; mixed %.1f = %.2fx FP64 %.1f, dfloat %.1f; "
                       "max backward error mixed %.1e, fp64 %.1e; corrections %.0f and FP64 "
                       "re-solves %.0f per mixed step"
                       % (headp, head["value"], mx["value"], line["mixed_speedup_vs_fp64"],
                          res["fp64"]["value"], res["dfloat"]["value"], mx["max_backward_error"],
                          res["fp64"]["max_backward_error"], mx["corrections_per_step"],
                          mx["fp64_resolves_per_step"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
