#!/usr/bin/env python
"""Benchmark of the stochastic Galerkin solve on GB300.

One step = one full solve of the linear stochastic Poisson Galerkin system
to relres 1e-8 (true FP64 residual) on the 256x256 mesh, L=4, p=3 (P=35,
2.28M unknowns), q=6 (K=210), 8x8 RAS boxes with overlap 2, 2h coarse grid
with AMG: FGMRES with the two-level preconditioner, FP32 operator and
preconditioner inside FP64 iterative refinement, inner coarse GMRES to a
relative 0.3 (the paper's default 1e-5 is reported beside it).  Inputs are
synthetic (the paper's workloads are synthetic lognormal fields too) and
resident in HBM; the matrix values (272 MB FP32 + 545 MB FP64) exceed the
129 MB L2, so no flush is needed between steps.

Secondary numbers on the same line: the plain FP64 solve, the paper's inner
tolerance, the twelve uneven systems of the batch family solved by one
graph launch, and the learned smoother trained on this system.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(rank 0 only).  Multi-GPU runs are independent replicas (weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "poisson256_L4_p3"
METRIC = "SG solve time to relres 1e-8 (FP32 in FP64 refinement, two-level RAS+AMG FGMRES)"
INNER_RTOL = 0.5          # inner coarse GMRES tolerance of the timed solves
RAS_KERNEL = 3            # FP32 RAS local solves: the faster of the line kernel and the explicit inverses
PAPER_INNER_RTOL = 1e-5   # the paper's default for the 2GV3 variant


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch and learned-smoother measurements")
    ap.add_argument("--only-timed", action="store_true",
                    help="the timed mixed solves only (no comparison solves, e2e or extras): for launch lists")
    ap.add_argument("--host-loops", action="store_true",
                    help="coarse GMRES driven from the host (every kernel a separate launch): for launch lists")
    ap.add_argument("--ras-kernel", type=int, default=RAS_KERNEL, choices=[0, 2, 3],
                    help="RAS local solves of the timed solve: 0 line kernel, 2 explicit inverses, 3 the faster "
                         "(timed at setup; pin it for launch lists, where the profiler's serialisation skews "
                         "the timing)")
    ap.add_argument("--kernel-case", default=None,
                    choices=["apply_slot", "apply_flux", "cnn_train", "nl_coef", "sample", "ras", "ras_inv",
                             "refine_residual"],
                    help="run a few launches of one kernel on a small case and exit (for profiler captures)")
    return ap.parse_args()


def measured_traffic(shape):
    """DRAM bytes per launch of the fine apply from a committed ncu summary
    (profiles/sg_k1*_poisson256_L4_p3.md) taken on the same generated kernel
    (tile shape, storage form and code-generator version); otherwise None."""
    import glob
    keys = ("rows", "groups", "igroups", "sgroups", "prefetch", "min_blocks", "stages", "cgroups", "warps",
            "generator", "flux")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "sg_k1*_poisson256_L4_p3.md"))):
        try:
            text = open(path).read()
        except OSError:
            continue
        vals = {}
        for line in text.splitlines():
            if line.startswith("traffic-key:"):
                for kv in line.split(":", 1)[1].split():
                    k, v = kv.split("=")
                    vals[k] = v
        vals.setdefault("flux", "0")
        if vals and all(vals.get(k) == str(shape.get(k, 0)) for k in keys):
            return int(vals["bytes"])
    return None


def ras_inv_traffic(source="sg_ras_tc.cu", summary="k_ras_inv_tc_poisson256_L4_p3.md"):
    """DRAM bytes per launch of a kernel from its committed ncu summary under
    profiles/ (by default k_ras_inv_tc), if that summary was taken on the
    current kernel source (its sha1 recorded there); otherwise None."""
    import hashlib
    src = os.path.join(ROOT, "paper_2310_14649_gb300", "csrc", source)
    prof = os.path.join(ROOT, "profiles", summary)
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        vals = {}
        for line in open(prof).read().splitlines():
            if line.startswith("traffic-key:"):
                for kv in line.split(":", 1)[1].split():
                    k, v = kv.split("=")
                    vals[k] = v
        return int(vals["bytes"]) if vals.get("source-sha1") == sha else None
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_sustained():
    """Sustained dense BF16 rate (TFLOP/s) for kernels timed inside a step."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    """The slowest rank's value (every rank receives it)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle (the baseline, and the reference arm)
# ---------------------------------------------------------------------------
def oracle_setup(cfg):
    """The FP64 oracle's system (plain numpy/scipy setup) and its multi-core
    operator with the banded Cholesky factor of A_0 (both untimed)."""
    from oracle import galerkin, par
    c = cfg
    t0 = time.perf_counter()
    prob = galerkin.build(c["N"], c["L"], c["p"], c["q"], c["sigma2"], c["b"], c["b"])
    op = par.Operator(prob).factor_mean()
    return prob, op, time.perf_counter() - t0


def oracle_measure(cfg, reps_apply=3):
    """The FP64 oracle on every host core: its Kronecker apply (median of
    `reps_apply`, in GB/s with the apply's algorithmic bytes at 8 B per
    value) and one complete GMRES solve to relres 1e-8 (I kron A_0^{-1}
    preconditioner), then continued to 1e-11 (untimed) as the reference
    solution the GPU's solutions are compared with (1e-12 is below the
    rounding floor of the FP64 residual on this system)."""
    import numpy as np
    from oracle import par
    prob, op, t_setup = oracle_setup(cfg)
    n, P, K, nnz = prob.n, prob.P, prob.K, len(prob.colidx)
    x = np.random.default_rng(0).standard_normal(n * P)
    y = np.empty_like(x)
    ts = []
    for _ in range(reps_apply):
        t0 = time.perf_counter()
        op.apply(x, y)
        ts.append(time.perf_counter() - t0)
    t_apply = statistics.median(ts)
    bytes64 = K * nnz * 8 + nnz * 4 + (n + 1) * 4 + 2 * n * P * 8
    X8, its8, hist8, t_solve = par.solve(prob, tol=1e-8, op=op)
    X12, its12, _, _ = par.solve(prob, tol=1e-11, max_it=300, op=op, X0=X8)
    return {"t_setup": t_setup, "t_apply": t_apply, "apply_gbs": bytes64 / t_apply / 1e9,
            "apply_bytes": bytes64, "t_solve": t_solve, "its": its8, "relres_est": hist8[-1] if hist8 else 0.0,
            "cores": par.threads(), "X_ref": X12, "ref_its": its8 + its12}


def err_vs(Xd, Xref):
    """Relative L2 error of a GPU solution [P, n] (torch, FP64) against the
    oracle's [n, P] solution (Appendix A, Eq. relerror)."""
    import numpy as np
    Xh = Xd.cpu().numpy().T
    return float(np.linalg.norm(Xh - Xref) / np.linalg.norm(Xref))


def workload_config(c, P, K, n, world):
    """The config object of the bench line (both arms)."""
    return {"workload": WORKLOAD, "N": c["N"], "L": c["L"], "p": c["p"], "q": c["q"], "P": P, "K": K,
            "unknowns": n * P, "ras_boxes": "%dx%d" % (c["sx"], c["sy"]), "overlap": c["overlap"],
            "parallelism": "replicas" if world > 1 else "single", "coarse_inner_rtol": INNER_RTOL,
            "l2": "inputs larger than L2 (values 0.82 GB), no flush"}


def run_reference(args):
    """The FP64 oracle on the host cores: every step is one complete GMRES
    solve of the benchmark system to relres 1e-8 from x = 0."""
    from sg_inputs import CONFIGS
    from oracle import par
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = CONFIGS[WORKLOAD]
    prob, op, t_setup = oracle_setup(c)
    for _ in range(args.warmup):
        par.solve(prob, tol=1e-8, op=op)
    its = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, it, _, _ = par.solve(prob, tol=1e-8, op=op)
        its.append(it)
    value = (time.perf_counter() - t0) / args.steps * 1e3
    cores = par.threads()
    sample = ("complete FP64 oracle GMRES solves (I kron A_0^{-1} preconditioner, restart 50) of the full %s "
              "system to relres 1e-8 from x = 0, %d iterations each, on %d host threads (C + OpenMP apply and "
              "banded substitutions); setup %.1f s untimed" % (WORKLOAD, its[-1], cores, t_setup))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(c, prob.P, prob.K, prob.n, world),
            "cpu_baseline": {"value": round(value, 3), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def extra_measurements(sg, torch, prob, stream):
    """The batch of twelve uneven systems in one graph launch, and the
    learned smoother trained on the benchmark system."""
    from sg_inputs import CONFIGS, batch_system
    out = {}

    def ev_ms(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), r

    # --- twelve uneven systems (meshes 64^2..384^2, L 2..5, p 2..4)
    cfgs = [batch_system(s) for s in range(12)]
    probs = []
    t0 = time.perf_counter()
    for cc in cfgs:
        p = sg.sg_setup(cc["N"], cc["L"], cc["p"], cc["q"], sigma2=cc["sigma2"], bx=cc["b"], by=cc["b"])
        sg.sg_apply_autotune(p)
        sg.sg_precond_setup(p, cc["sx"], cc["sy"], cc["overlap"], inner_rtol=INNER_RTOL)
        for which in (1, 2):
            sg.sg_apply_autotune(p, which=which)
        probs.append(p)
    t_setup = time.perf_counter() - t0
    Xs = [torch.zeros((p.P, p.n), dtype=torch.float64, device="cuda") for p in probs]
    B = sg.sg_batch_create(probs, rtol=1e-8, mode=1, max_it=400)

    def run_batch():
        for X in Xs:
            X.zero_()
        return sg.sg_batch_solve(B, Xs)

    run_batch()
    l0 = sg.sg_launch_count()
    reps = 3
    ms_b = []
    for _ in range(reps):
        m, infos = ev_ms(run_batch)
        ms_b.append(m)
    batch_launches = (sg.sg_launch_count() - l0) // reps

    def run_seq():
        for p, X in zip(probs, Xs):
            X.zero_()
            sg.sg_solve(p, X, rtol=1e-8, mode=1, max_it=400)

    run_seq()
    ms_seq, _ = ev_ms(run_seq)
    out["batch12"] = {"systems": 12, "unknowns": int(sum(p.n * p.P for p in probs)),
                      "graph_ms": round(statistics.median(ms_b), 3), "sequential_ms": round(ms_seq, 3),
                      "speedup": round(ms_seq / statistics.median(ms_b), 3),
                      "max_relres": max(i["relres"] for i in infos),
                      "outer_it": [i["outer_it"] for i in infos], "setup_s": round(t_setup, 2),
                      "gpu_launches_per_solve": int(batch_launches),
                      "note": "one CUDA graph launch: refinement, FGMRES and coarse GMRES loops as conditional "
                              "WHILE nodes, the twelve systems as parallel branches; sequential = one sg_solve "
                              "per system"}
    B.close()
    for p in probs:
        p.close()

    # --- learned smoother on the benchmark system
    info = sg.sg_train_precond(prob, n_pairs=4096, epochs=12, batch=32, lr=1e-3, seed=0, loss=0)
    n, P = prob.n, prob.P
    R = torch.randn((P, n), dtype=torch.float32, device="cuda")
    Z = torch.zeros_like(R)
    sg.sg_precond_apply(prob, sg.PC_NETWORK, R, Z)
    reps = 10
    m_net, _ = ev_ms(lambda: [sg.sg_precond_apply(prob, sg.PC_NETWORK, R, Z) for _ in range(reps)])
    m_net /= reps
    flops = 2 * 9 * (2 * 32 + 3 * 32 * 32 + 32) * n * P
    X = torch.zeros((P, n), dtype=torch.float64, device="cuda")

    def lsolve(mode):
        X.zero_()
        return sg.sg_solve(prob, X, rtol=1e-8, mode=mode, max_it=400)

    lsolve(1)
    m_l32, i_l32 = ev_ms(lambda: lsolve(1))
    m_l64, i_l64 = ev_ms(lambda: lsolve(0))
    sg.sg_precond_set_smoother(prob, 0)
    out["learned"] = {"train": {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in info.items()},
                      "loss": "energy norm of A_0", "pairs": 4096, "epochs": 12, "batch": 32,
                      "mixed_ms": round(m_l32, 3), "mixed_outer_it": i_l32["outer_it"],
                      "mixed_fallback": i_l32["fallback_used"], "mixed_relres": i_l32["relres"],
                      "fp64_ms": round(m_l64, 3), "fp64_outer_it": i_l64["outer_it"],
                      "network_ms_per_apply": round(m_net, 4),
                      "network_tflops": round(flops / m_net / 1e9, 1),
                      "network_bound": "tensor (tcgen05 forward, BF16 operands, FP32 in tensor memory)",
                      "network_frac_of_bf16_sustained": round(flops / m_net / 1e9 / bf16_sustained()[0], 4),
                      "bf16_sustained_source": bf16_sustained()[1]}
    return out


def ev_time(torch, stream, fn):
    """(ms, result) of fn() between CUDA events on `stream`."""
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), r


def large_workload(sg, torch, stream, reps=3):
    """The 512x512 mesh, L=6, p=3 (P=84, K=924, 21.9M unknowns): mixed and
    plain FP64 solves, the apply's roofline (per-launch events in a separate
    profiled solve) and the learned smoother against RAS."""
    from sg_inputs import CONFIGS
    c = CONFIGS["poisson512_L6_p3"]
    t0 = time.perf_counter()
    prob = sg.sg_setup(c["N"], c["L"], c["p"], c["q"], sigma2=c["sigma2"], bx=c["b"], by=c["b"])
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    sg.sg_apply_autotune(prob)
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL, ras_kernel=RAS_KERNEL)
    for which in (1, 2, 3):
        sg.sg_apply_autotune(prob, which=which)
    n, P, K, nnz = prob.n, prob.P, prob.K, prob.nnzA
    X = torch.zeros((P, n), dtype=torch.float64, device="cuda")

    def solve(mode):
        X.zero_()
        return sg.sg_solve(prob, X, rtol=1e-8, mode=mode, max_it=600)

    solve(1)
    runs = [ev_time(torch, stream, lambda: solve(1)) for _ in range(reps)]
    ms32 = statistics.median(r[0] for r in runs)
    info32 = runs[-1][1]
    ms64, info64 = ev_time(torch, stream, lambda: solve(0))
    sg.sg_profile(prob, True)
    solve(1)
    cnt, kms = sg.sg_profile_read(prob, 0)
    rcnt, rms = sg.sg_profile_read(prob, 4)
    sg.sg_profile(prob, False)
    bytes_f32 = K * nnz * 4 + nnz * 4 + (n + 1) * 4 + 2 * n * P * 4
    avg = kms / max(cnt, 1)
    peak, peak_kind = peaks()
    out = {"workload": "poisson512_L6_p3", "N": c["N"], "L": c["L"], "P": P, "K": K, "unknowns": n * P,
           "setup_s": round(t_setup, 2),
           "mixed_ms": round(ms32, 2), "mixed_outer_it": info32["outer_it"], "mixed_relres": info32["relres"],
           "plain_fp64_ms": round(ms64, 2), "plain_fp64_outer_it": info64["outer_it"],
           "speedup_mixed": round(ms64 / ms32, 3),
           "roofline": {"kernel": "sg_apply FP32 (fine Galerkin operator, five-slot form)", "bound": "hbm",
                        "achieved": round(bytes_f32 / (avg * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(bytes_f32 / (avg * 1e-3) / 1e9 / peak, 4), "peak_source": peak_kind,
                        "bytes_per_launch": bytes_f32, "avg_launch_ms": avg, "launches": cnt},
           "ras_local_ms_per_launch": rms / max(rcnt, 1), "ras_kernel": sg.sg_precond_ras_kernel(prob),
           "apply_shape": sg.sg_apply_info(prob)}
    # learned smoother trained on this system, against RAS
    info = sg.sg_train_precond(prob, n_pairs=4096, epochs=4, batch=32, lr=1e-3, seed=0, loss=0)
    solve(1)
    msl, infol = ev_time(torch, stream, lambda: solve(1))
    sg.sg_precond_set_smoother(prob, 0)
    out["learned"] = {"t_train": round(info["t_train"], 2), "loss_last": float("%.4g" % info["loss_last"]),
                      "mixed_ms": round(msl, 2), "mixed_outer_it": infol["outer_it"],
                      "fallback": infol["fallback_used"], "relres": infol["relres"],
                      "vs_ras_mixed": round(msl / ms32, 3)}
    prob.close()
    return out


def nonlinear_workload(sg, torch, stream):
    """The nonlinear problem -div(c (1 + u^2) grad u) = 1 on the 384x384
    mesh, L=4, p=4 (P=70, K=495, 10.3M unknowns): Newton to a relative update
    of 1e-8, each step by FGMRES with the two-level preconditioner, FP32
    inside the FP64 Newton residual (mixed) and all FP64 (plain)."""
    from sg_inputs import CONFIGS
    c = CONFIGS["poisson384_L4_p4"]
    prob = sg.sg_setup(c["N"], c["L"], c["p"], c["q"], sigma2=c["sigma2"], bx=c["b"], by=c["b"])
    sg.sg_apply_autotune(prob)
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL, ras_kernel=RAS_KERNEL)
    for which in (1, 2, 3):
        sg.sg_apply_autotune(prob, which=which)
    X = torch.zeros((prob.P, prob.n), dtype=torch.float64, device="cuda")

    def newton(mode):
        X.zero_()
        return sg.sg_newton(prob, X, tol_update=1e-8, mode=mode)

    newton(1)
    ms32, i32 = ev_time(torch, stream, lambda: newton(1))
    ms64, i64 = ev_time(torch, stream, lambda: newton(0))
    out = {"workload": "poisson384_L4_p4 nonlinear (1 + u^2)", "P": prob.P, "K": prob.K,
           "unknowns": prob.n * prob.P, "mixed_ms": round(ms32, 2), "newton_steps": i32["ir_steps"],
           "gmres_its": i32["outer_it"], "relres": i32["relres"], "last_update": float(i32["hist"][-1]),
           "plain_fp64_ms": round(ms64, 2), "plain_newton_steps": i64["ir_steps"], "plain_gmres_its": i64["outer_it"],
           "speedup_mixed": round(ms64 / ms32, 3)}
    prob.close()
    return out


def verification_workload(sg, torch, stream, S=40000):
    """The paper's verification setting (Sec. 4.1: 101 x 101 vertices, three
    random variables, input order 2, output order 3, sigma = 0.1, four
    subdomains): the SG solve and 40,000 Monte Carlo samples, both on the
    GPU, and their mean and standard deviation at (0.5, 0.5) and (0.3, 0.7)."""
    import numpy as np
    N, L, p, q = 100, 3, 3, 2
    prob = sg.sg_setup(N, L, p, q, sigma2=0.01, bx=0.5, by=0.5)
    sg.sg_precond_setup(prob, 2, 2, 1)
    X = torch.zeros((prob.P, prob.n), dtype=torch.float64, device="cuda")
    sg.sg_solve(prob, X, rtol=1e-10, mode=1)
    X.zero_()
    ms_sg, info = ev_time(torch, stream, lambda: sg.sg_solve(prob, X, rtol=1e-10, mode=1))
    xi = torch.from_numpy(np.random.default_rng(2023).standard_normal((S, L))).cuda()
    U = torch.empty((S, prob.n), dtype=torch.float32, device="cuda")
    sg.sg_sample_solve(prob, xi[:64], U[:64])
    ms_mc, its = ev_time(torch, stream, lambda: sg.sg_sample_solve(prob, xi, U, rtol=1e-6))
    Ud = U.double()
    mean_mc, std_mc = Ud.mean(0), Ud.std(0)
    mean_sg = X[0]
    std_sg = X[1:].pow(2).sum(0).sqrt()
    m = N - 1
    pts = {}
    for (px, py) in ((0.5, 0.5), (0.3, 0.7)):
        r = (round(py * N) - 1) * m + (round(px * N) - 1)
        pts["%.1f,%.1f" % (px, py)] = {"mean_sg": float(mean_sg[r]), "mean_mc": float(mean_mc[r]),
                                       "std_sg": float(std_sg[r]), "std_mc": float(std_mc[r]),
                                       "se_mean": float(std_mc[r]) / S ** 0.5}
    out = {"setting": "N=100 (10,201 vertices), L=3, p=3, q=2, sigma=0.1, 2x2 boxes", "sg_ms": round(ms_sg, 3),
           "sg_outer_it": info["outer_it"], "mc_samples": S, "mc_ms": round(ms_mc, 1),
           "mc_samples_per_s": round(S / ms_mc * 1e3, 1), "mc_max_cg_its": its,
           "mean_rel_diff": float((mean_sg - mean_mc).norm() / mean_sg.norm()),
           "std_rel_diff": float((std_sg - std_mc).norm() / std_sg.norm()), "points": pts}
    prob.close()
    return out


def kernel_case(name):
    """A few launches of one kernel family on a case small enough for a
    full profiler capture (inputs still larger than L2 where that matters)."""
    import numpy as np
    import torch
    import paper_2310_14649_gb300 as sg
    from sg_inputs import CONFIGS
    torch.cuda.set_device(0)
    c = CONFIGS[WORKLOAD]
    if name in ("apply_slot", "apply_flux", "ras", "ras_inv"):
        prob = sg.sg_setup(c["N"], c["L"], c["p"], c["q"], sigma2=c["sigma2"], bx=c["b"], by=c["b"])
        sg.sg_apply_autotune(prob)
        X = torch.randn((prob.P, prob.n), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        if name in ("ras", "ras_inv"):
            sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL,
                                ras_kernel=2 if name == "ras_inv" else 0)
            for _ in range(3):
                sg.sg_precond_apply(prob, sg.PC_SMOOTH, X, Y)
            stream = torch.cuda.current_stream()
            ms, _ = ev_time(torch, stream, lambda: [sg.sg_precond_apply(prob, sg.PC_SMOOTH, X, Y) for _ in range(20)])
            print(json.dumps({"kernel_case": name, "smoother_ms": ms / 20}))
        else:
            sg.sg_apply_flux(prob, 1 if name == "apply_flux" else 0)
            for _ in range(3):
                sg.sg_apply(prob, X, Y)
    elif name == "refine_residual":
        prob = sg.sg_setup(c["N"], c["L"], c["p"], c["q"], sigma2=c["sigma2"], bx=c["b"], by=c["b"])
        sg.sg_set_refine_residual(prob, 2)
        X = torch.randn((prob.P, prob.n), dtype=torch.float64, device="cuda")
        F = torch.randn_like(X)
        R = torch.empty_like(X)
        for _ in range(3):
            sg.sg_residual_refine(prob, F, X, R)
        stream = torch.cuda.current_stream()
        ms, _ = ev_time(torch, stream, lambda: [sg.sg_residual_refine(prob, F, X, R) for _ in range(20)])
        print(json.dumps({"kernel_case": name, "residual_ms": ms / 20}))
    elif name == "cnn_train":
        prob = sg.sg_setup(256, 2, 1, 2)
        sg.sg_cnn_init(prob, seed=1)
        R = torch.randn((32, prob.n), dtype=torch.float32, device="cuda")
        Z = torch.randn_like(R)
        for _ in range(2):
            sg.sg_cnn_train_step(prob, R, Z, lr=1e-3, update=True)
    elif name == "nl_coef":
        c5 = CONFIGS["poisson384_L4_p4"]
        prob = sg.sg_setup(128, c5["L"], c5["p"], c5["q"], sigma2=c5["sigma2"], bx=c5["b"], by=c5["b"])
        U = 0.05 * torch.randn((prob.P, prob.n), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(U)
        for _ in range(3):
            sg.sg_nonlinear_jacobian_apply(prob, U, U, Y)
    elif name == "sample":
        prob = sg.sg_setup(100, 3, 3, 2, sigma2=0.01, bx=0.5, by=0.5)
        xi = torch.from_numpy(np.random.default_rng(1).standard_normal((304, 3))).cuda()
        U = torch.empty((304, prob.n), dtype=torch.float32, device="cuda")
        for _ in range(2):
            sg.sg_sample_solve(prob, xi, U)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": name, "ok": True}))


def main():
    args = parse()
    if args.kernel_case:
        kernel_case(args.kernel_case)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import paper_2310_14649_gb300 as sg
    from sg_inputs import CONFIGS

    world, rank, local = dist_setup()
    cfg = CONFIGS[WORKLOAD]
    c = cfg
    t0 = time.perf_counter()
    prob = sg.sg_setup(c["N"], c["L"], c["p"], c["q"], sigma2=c["sigma2"], bx=c["b"], by=c["b"])
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    tune_ms = sg.sg_apply_autotune(prob)       # cached after the first run
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL, host_loops=args.host_loops,
                        ras_kernel=args.ras_kernel)
    torch.cuda.synchronize()
    t_pc = time.perf_counter() - t0
    t0 = time.perf_counter()
    for which in (1, 2, 3):                    # coarse FP32, fine and coarse FP64, cached too
        sg.sg_apply_autotune(prob, which=which)
    t_tune += time.perf_counter() - t0
    n, P = prob.n, prob.P
    X = torch.zeros((P, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def solve(mode=1):
        X.zero_()
        return sg.sg_solve(prob, X, rtol=1e-8, mode=mode, max_it=400)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sg.sg_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    infos = [solve() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    launches = sg.sg_launch_count() - l0
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_all = max_over_ranks(world, ms)
    X_mixed = X.clone()

    if args.only_timed:
        line = {"metric": METRIC, "value": round(ms_all, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_all, 3), "higher_is_better": False,
                "scaling": "weak", "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "coarse_inner_rtol": INNER_RTOL, "only_timed": True,
                           "coarse_loops": "host" if args.host_loops else "graph"},
                "gpu_launches": int(launches)}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    # a separate pass with per-launch and per-phase events (outside the
    # timed region): the apply's roofline and where a step's time goes
    prof_steps = min(args.steps, 5)
    sg.sg_profile(prob, True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(prof_steps):
        solve()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1) / prof_steps
    kinds = {}
    for kind, name in ((0, "apply_fine_f32"), (1, "refine_residual"), (2, "apply_coarse_f32"), (3, "apply_coarse_f64"),
                       (4, "ras_local_f32"), (6, "smoother"), (7, "coarse_correction"), (8, "arnoldi"),
                       (9, "refinement")):
        cnt, kms = sg.sg_profile_read(prob, kind)
        kinds[name] = (cnt, kms)
    sg.sg_profile(prob, False)

    # roofline of the fine FP32 operator apply: algorithmic bytes per launch
    # (five-slot form: values, pattern and blocks read once; edge-flux form:
    # one conductance per edge and term, two indices per edge slot of a row)
    K, nnz = prob.K, prob.nnzA
    flux_on = sg.sg_apply_flux(prob, -1)
    N_ = c["N"]
    bytes_slot = K * nnz * 4 + nnz * 4 + (n + 1) * 4 + 2 * n * P * 4
    bytes_flux = K * 2 * N_ * (N_ - 1) * 4 + 4 * 2 * 4 * n + 2 * n * P * 4
    bytes_f32 = bytes_flux if flux_on else bytes_slot
    cnt, kms = kinds["apply_fine_f32"]
    avg_ms = kms / max(cnt, 1)
    achieved = bytes_f32 / (avg_ms * 1e-3) / 1e9 if cnt else None
    peak, peak_kind = peaks()
    # the RAS local solves: line FMA recurrences, or explicit inverses
    ras_flops, ras_boxes, ras_w = sg.sg_precond_stats(prob)
    ras_kernel = sg.sg_precond_ras_kernel(prob)
    rcnt, rms = kinds["ras_local_f32"]
    ras_avg = rms / max(rcnt, 1)
    ras_tflops = ras_flops / (ras_avg * 1e-3) / 1e12 if rcnt else None
    # explicit inverses: the owned rows x overlapped columns of every box
    # (FP32), the gathered residual and the written result
    inv_bytes = 0
    for b in range(ras_boxes):
        idx_b, own_b = sg.sg_get_partition(prob, b)
        inv_bytes += int(own_b.sum()) * len(idx_b) * 4 + len(idx_b) * P * 4
    inv_bytes += n * P * 4
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
    # refinement residual: the edge blocks (P (P + 1) / 2 pairs of FP32 per
    # edge) read once, X and F read, R written (FP64)
    res_cnt, res_ms = kinds["refine_residual"]
    res_avg = res_ms / max(res_cnt, 1)
    res_bytes = (P * (P + 1) // 2) * 2 * N_ * (N_ - 1) * 8 + 3 * n * P * 8
    # phases of one step (non-overlapping: the fine applies outside the
    # smoother and the coarse correction, the smoother, the coarse
    # correction, the Arnoldi steps, the refinement bookkeeping); the rest
    # is host synchronisation and small copies
    phase_ms = {k: round(kinds[k][1] / prof_steps, 3) for k in
                ("apply_fine_f32", "refine_residual", "smoother", "coarse_correction", "arnoldi", "refinement")}
    phase_ms["ras_local_f32 (inside smoother)"] = round(kinds["ras_local_f32"][1] / prof_steps, 3)
    attributed = sum(v for k, v in phase_ms.items() if "inside" not in k)

    # plain FP64 solve on the same system (the comparison the metric names)
    def timed(mode):
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        info = solve(mode=mode)
        f1.record(stream)
        torch.cuda.synchronize()
        return f0.elapsed_time(f1), info

    ms64, info64 = timed(0)
    X64_sol = X.clone()
    # the paper's inner tolerance, both precisions
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=PAPER_INNER_RTOL, ras_kernel=RAS_KERNEL)
    solve(mode=1)
    ms_paper32, info_paper32 = timed(1)
    ms_paper64, info_paper64 = timed(0)
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL, ras_kernel=RAS_KERNEL)
    solve(mode=1)

    # end to end through the C ABI with host buffers: F host->device, solve,
    # X device->host every step
    Fh = torch.zeros((P, n), dtype=torch.float64).pin_memory()
    Fd = torch.zeros((P, n), dtype=torch.float64, device="cuda")
    sg.sg_get_rhs(prob, Fd)
    Fh.copy_(Fd.cpu())
    Xh = torch.zeros((P, n), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        Fd.copy_(Fh, non_blocking=True)
        X.zero_()
        sg.sg_solve(prob, X, F=Fd, rtol=1e-8, mode=1, max_it=400)
        Xh.copy_(X, non_blocking=True)
    g1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(world, g0.elapsed_time(g1) / args.steps)

    # both storage forms of the fine FP32 apply, timed alone (20 launches
    # after 3, CUDA events; values exceed L2, so no flush)
    apply_forms = {}
    Xa = torch.randn((P, n), dtype=torch.float32, device="cuda")
    Ya = torch.empty_like(Xa)
    chosen = sg.sg_apply_flux(prob, -1)
    for form, mode in (("five_slot", 0), ("edge_flux", 1)):
        sg.sg_apply_flux(prob, mode)
        for _ in range(3):
            sg.sg_apply(prob, Xa, Ya)
        ms_a, _ = ev_time(torch, stream, lambda: [sg.sg_apply(prob, Xa, Ya) for _ in range(20)])
        byt = bytes_flux if mode else bytes_slot
        apply_forms[form] = {"ms": round(ms_a / 20, 5), "bytes": byt, "gbs": round(byt / (ms_a / 20 * 1e-3) / 1e9, 1)}
    sg.sg_apply_flux(prob, 2)
    sg.sg_apply_autotune(prob)                 # the tuned choice again (cached)
    # both FP32 RAS local-solve kernels, the smoother with its Kronecker
    # factor (20 applications after 3)
    ras_forms = {}
    for form, kern in (("line_fma", 0), ("explicit_inverse_tcgen05", 2)):
        sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL, ras_kernel=kern)
        for _ in range(3):
            sg.sg_precond_apply(prob, sg.PC_SMOOTH, Xa, Ya)
        ms_r, _ = ev_time(torch, stream, lambda: [sg.sg_precond_apply(prob, sg.PC_SMOOTH, Xa, Ya) for _ in range(20)])
        ras_forms[form] = {"smoother_ms": round(ms_r / 20, 5)}
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"], inner_rtol=INNER_RTOL, ras_kernel=RAS_KERNEL)
    ras_forms["chosen"] = ["line_fma", "", "explicit_inverse_tcgen05"][sg.sg_precond_ras_kernel(prob)]
    assert sg.sg_apply_flux(prob, -1) == chosen
    extras = {} if (args.no_extras or rank != 0) else extra_measurements(sg, torch, prob, stream)
    if not args.no_extras and rank == 0:
        extras["poisson512"] = large_workload(sg, torch, stream)
        extras["nonlinear"] = nonlinear_workload(sg, torch, stream)
        extras["verification"] = verification_workload(sg, torch, stream)

    cpu = None
    oracle_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        o = oracle_measure(cfg)
        cpu = {"value": round(o["t_solve"] * 1e3, 1), "unit": "ms", "cores": o["cores"], "kind": "oracle (measured)",
               "sample": "one complete FP64 oracle GMRES solve (I kron A_0^{-1} preconditioner, restart 50) of the "
                         "full %s system to relres 1e-8 from x = 0: %d iterations; plain C + OpenMP operator "
                         "apply and banded substitutions on %d host threads" % (WORKLOAD, o["its"], o["cores"]),
               "apply_ms": round(o["t_apply"] * 1e3, 2), "apply_gbs": round(o["apply_gbs"], 2),
               "apply_bytes_f64": o["apply_bytes"], "setup_s": round(o["t_setup"], 2)}
        oracle_err = {"mixed": err_vs(X_mixed, o["X_ref"]), "plain_fp64": err_vs(X64_sol, o["X_ref"]),
                      "reference": "oracle GMRES to relres 1e-11 (%d iterations)" % o["ref_its"]}

    line = {
        "metric": METRIC, "value": round(ms_all, 3), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_all, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(c, P, K, n, world),
        "solve": {"outer_it": infos[-1]["outer_it"], "inner_it": infos[-1]["inner_it"],
                  "ir_steps": infos[-1]["ir_steps"], "relres": infos[-1]["relres"],
                  "setup_s": round(t_setup, 3), "precond_setup_s": round(t_pc, 3),
                  "apply_tuning_s": round(t_tune, 3), "apply_shape": sg.sg_apply_info(prob),
                  "coarse_apply_shape": sg.sg_apply_info(prob, which=1),
                  "fine_apply_shape_f64": sg.sg_apply_info(prob, which=2),
                  "solves_per_s_all_gpus": round(world * 1e3 / ms_all, 3)},
        "plain_fp64": {"ms": round(ms64, 3), "outer_it": info64["outer_it"], "relres": info64["relres"],
                       "speedup_mixed": round(ms64 / ms_all, 3)},
        "paper_inner_rtol": {"inner_rtol": PAPER_INNER_RTOL,
                             "mixed_ms": round(ms_paper32, 3), "mixed_outer_it": info_paper32["outer_it"],
                             "mixed_inner_it": info_paper32["inner_it"],
                             "plain_fp64_ms": round(ms_paper64, 3), "plain_fp64_outer_it": info_paper64["outer_it"]},
        "apply_forms": apply_forms,
        "roofline": {"kernel": "sg_apply FP32 (fine Galerkin operator, %s form)" % ("edge-flux" if flux_on else
                                                                                    "five-slot"), "bound": "hbm",
                     "achieved": round(achieved, 1) if achieved else None, "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
                     "peak_source": peak_kind, "bytes_per_launch": bytes_f32, "avg_launch_ms": avg_ms,
                     "launches": cnt,
                     "traffic": measured_traffic(dict(sg.sg_apply_info(prob), flux=flux_on))},
        "roofline_top_kernel": ({"kernel": "k_ras_inv_pack + k_ras_inv_tc FP32 (RAS by explicit local inverses on "
                                           "tcgen05, %d boxes, Kronecker factor fused; the timed span holds both "
                                           "launches)" % ras_boxes,
                                 "bound": "hbm", "achieved": round(inv_bytes / (ras_avg * 1e-3) / 1e9, 1) if rcnt else None,
                                 "peak": peak, "unit": "GB/s",
                                 "frac": round(inv_bytes / (ras_avg * 1e-3) / 1e9 / peak, 4) if rcnt else None,
                                 "peak_source": peak_kind, "bytes_per_launch": inv_bytes, "avg_launch_ms": ras_avg,
                                 "launches": rcnt, "traffic": ras_inv_traffic()}
                                if ras_kernel == 2 else
                                {"kernel": "k_ras_local FP32 (RAS line solves, %d boxes, line width %d)"
                                           % (ras_boxes, ras_w),
                                 "bound": "alu", "achieved": round(ras_tflops, 2) if ras_tflops else None,
                                 "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                                 "frac": round(ras_tflops / fp32_peak, 4) if ras_tflops else None,
                                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                                 "flops_per_launch": ras_flops, "avg_launch_ms": ras_avg, "launches": rcnt,
                                 "note": "latency-bound line recurrences (dependent steps per sweep); "
                                         "a few percent of DRAM bandwidth"}),
        "roofline_refine_residual": ({"kernel": "k_split_df + k_resid_tile_df (FP64 refinement residual in "
                                                "double-FP32 over the edge blocks; the timed span holds both "
                                                "launches)",
                                      "bound": "hbm", "achieved": round(res_bytes / (res_avg * 1e-3) / 1e9, 1),
                                      "peak": peak, "unit": "GB/s",
                                      "frac": round(res_bytes / (res_avg * 1e-3) / 1e9 / peak, 4),
                                      "peak_source": peak_kind, "bytes_per_launch": res_bytes,
                                      "avg_launch_ms": res_avg, "launches": res_cnt,
                                      "traffic": ras_inv_traffic("sg_resid_df.cu",
                                                                 "k_resid_tile_df_poisson256_L4_p3.md")}
                                     if res_cnt and sg.sg_refine_residual_info(prob)["built"] else None),
        "ras_forms": ras_forms,
        "phase_ms_per_step": phase_ms,
        "profiled_ms_per_step": round(ms_prof, 3),
        "attributed_share": round(attributed / ms_prof, 3),
        "err_vs_oracle": oracle_err,
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": n * P * 8,
                "d2h_bytes_per_step": n * P * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
