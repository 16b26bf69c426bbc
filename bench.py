"""Benchmark: VIF negative log-likelihood evaluations per second on one GB300.

Workload (default): n = 500,000 points uniform on [0,1]^8, ARD squared-exponential
kernel (length scales log-uniform in [0.2, 2], variance 1, nugget 0.01), m = 500
k-means++ inducing points, m_v = 20 correlation neighbours.  One step = one
vif_nll evaluation (low-rank part A, residual Vecchia factors, [F z] Gram,
capacitance Cholesky and the scalar) on the mixed-precision path; the neighbour
sets are built once beforehand, as in the paper's likelihood timings (Sec. 7.4).
The float64 GPU path is timed beside it on the same neighbour sets.

--impl reference runs the float64 CPU oracle (the method as the paper writes it)
on a bounded sample of the same workload on the host cores.

Prints one JSON line (rank 0).
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
sys.path.insert(0, ROOT)

METRIC = "VIF NLL evals/s at n=500k (mixed-precision GPU path)"
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vif", choices=["vif", "reference"])
    ap.add_argument("--n", type=int, default=500_000)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-laplace", action="store_true")
    ap.add_argument("--laplace-n", type=int, default=200_000)
    ap.add_argument("--no-small", action="store_true", help="skip the C1/C2 block")
    ap.add_argument("--laplace-only", action="store_true",
                    help="run only the C4 Laplace block and print its JSON (for profiling the PCG kernels)")
    ap.add_argument("--batch", type=int, default=256,
                    help="also time N independent C5-style problems per CUDA graph replay (0: skip)")
    return ap.parse_args()


def workload(n):
    from paper_2507_05064_gb300 import synth
    t0 = time.time()
    P = synth.config3(n=n)
    return P, time.time() - t0


def config_dict(P, n_gpus):
    return {"workload": f"vif-nll-se-ard-n{P.X.shape[0]}-d8-m{P.Z.shape[0]}-mv{P.mv}",
            "n": int(P.X.shape[0]), "d": int(P.X.shape[1]), "m": int(P.Z.shape[0]), "m_v": int(P.mv),
            "kernel": "squared-exponential ARD", "nugget": P.theta.nugget,
            "l2": f"inputs larger than L2 (A alone is n*m*4 B = {P.X.shape[0] * P.Z.shape[0] * 4 / 1e9:.2f} GB)",
            "parallelism": f"replicas x{n_gpus}"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index=0):
        self.rows = []
        self.proc = None
        self.dev = dev_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """Largest value over all ranks (the timing rule: max over ranks); identity
    without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def stage_algorithmic(P, stage):
    """Algorithmic flops and HBM bytes of one launch of a stage of the mixed path (float32
    storage), as the method counts them (2 flops per FMA; one pass over each array):
      lowrank_A       m^2 n / 2 FMA (A = L_m^{-1} K_mn), write A (4 n m bytes)
      vecchia_factor  n m [(q+1)(q+2)/2 + q] FMA (residual Gram of [A_N; a_i] and the F row)
                      + n q^3 / 6 (the Cholesky), read A once and write [F z] (4 n fpad)
      gram_FtF        n (m+1)(m+2) / 2 FMA, read [F z] once."""
    n, m, q = P.X.shape[0], P.Z.shape[0], P.mv
    fpad = ((m + 1 + 63) // 64) * 64
    if stage == "lowrank_A":
        return 2.0 * n * m * (m + 1) / 2, 4.0 * n * m
    if stage == "vecchia_factor":
        fma = n * ((q + 1) * (q + 2) / 2 * m + q * m) + n * q ** 3 / 6
        return 2.0 * fma, 4.0 * n * m + 4.0 * n * fpad
    if stage == "gram_FtF":
        return 2.0 * n * (m + 1) * (m + 2) / 2, 4.0 * n * fpad
    return 0.0, 0.0


# DRAM bytes per point of the CUDA-core factor kernel (factor_kernel<float, 3>) from one ncu
# capture of this source at n = 100,000 (379.4 MB read + 203.1 MB written per launch); reported,
# scaled by n, only while the kernel's source file still has this digest
FACTOR_TRAFFIC = {"bytes_per_point": 5824.9, "source_sha256": "3296c39430878a27f9c9dcf496e5f641bad8211bc78080d9a5cdf87a68c997d4"}


def factor_traffic(n):
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_2507_05064_gb300", "csrc", "vif_factor.cu"), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return FACTOR_TRAFFIC["bytes_per_point"] * n if digest == FACTOR_TRAFFIC["source_sha256"] else None


def roofline_block(P, med, ms_step, pk, factor_path=1):
    """Roofline of the dense contractions (tensor-core bound) and of HBM, per stage and for the
    whole evaluation.  Each contraction is held to the tensor peak of the type it runs in:
    A (float16 split) and the tensor-core factor path at the measured dense bf16 burst peak
    (float16 has the same nominal rate), the Gram (tf32 split) at half of it (the nominal
    tf32 : bf16 ratio); the CUDA-core factor path is also held to the tf32 figure.  HBM is the
    measured copy bandwidth."""
    bf16 = pk.get("bf16_tflops")
    src = ("measured" if bf16 else "fallback")
    bf16 = bf16 or 1900.0
    hbm = pk.get("hbm_gbs") or 6800.0
    peak_of = {"lowrank_A": ("f16", bf16),
               "vecchia_factor": ("f16", bf16) if factor_path == 2 else ("tf32", bf16 / 2.0),
               "gram_FtF": ("tf32", bf16 / 2.0)}
    stages = {}
    tot_f = tot_b = t_tensor = 0.0
    for st in ("lowrank_A", "vecchia_factor", "gram_FtF"):
        f, b = stage_algorithmic(P, st)
        dt, pkt = peak_of[st]
        tot_f += f
        tot_b += b
        t_tensor += f / (pkt * 1e12)
        t = med[st] * 1e-3
        ff, fb = f / t / 1e12 / pkt, b / t / 1e9 / hbm
        stages[st] = {"ms": med[st], "tflops": f / t / 1e12, "tensor_dtype": dt, "peak_tflops": pkt,
                      "frac_tensor": ff, "gbs": b / t / 1e9, "frac_hbm": fb,
                      "binding": "tensor" if ff >= fb else "hbm", "frac": max(ff, fb),
                      "algorithmic_flops": f, "algorithmic_bytes": b}
    roof_ms = max(t_tensor, tot_b / (hbm * 1e9)) * 1e3
    dom = max(stages, key=lambda k: stages[k]["ms"])
    d = stages[dom]
    traffic = factor_traffic(P.X.shape[0]) if (dom == "vecchia_factor" and factor_path == 1) else None
    return {"kernel": dom, "bound": "tensor", "achieved": d["tflops"], "peak": d["peak_tflops"], "unit": "TFLOP/s",
            "frac": d["frac_tensor"], "traffic": traffic,
            "peak_source": (f"{d['tensor_dtype']}: {src} dense bf16 burst peak {bf16} TFLOP/s"
                            + (" x 1/2 (nominal tf32 : bf16)" if d["tensor_dtype"] == "tf32" else "")),
            "hbm_achieved_gbs": d["gbs"], "hbm_peak_gbs": hbm, "frac_hbm": d["frac_hbm"],
            "algorithmic_flops_per_launch": d["algorithmic_flops"],
            "algorithmic_bytes_per_launch": d["algorithmic_bytes"],
            "per_stage": stages,
            "whole_eval": {"algorithmic_flops": tot_f, "algorithmic_bytes": tot_b, "roofline_ms": roof_ms,
                           "ms": ms_step, "frac_whole_eval": roof_ms / ms_step}}


def launches_per_eval(m):
    """Kernel launches of one vif_nll call (counted from the launch sites; 169 for
    m = 500, as in the committed launch list)."""
    ch = lambda k: (k + 15) // 16      # 16 x 16 Cholesky tiles
    tr = (m + 31) // 32                # 32 x 32 triangular-inverse tiles
    nt, nt1 = ch(m), ch(m + 1)
    chol = lambda t: t + (t - 1)       # panel launches + trailing-update launches
    trtri = lambda t: 1 + 2 * (t - 1)  # diagonal tiles, then product + finish per block diagonal
    return (2 + 1 + chol(nt) + trtri(tr) + 2 + 1   # scaling x2, Sigma_m, Cholesky, inverse, L^-1 operand (row
                                                  # scales, tiles), A
            + 1 + 2 + 2 + chol(nt1) + 1)          # factor, Gram + reduce, logD sum, capacitance Cholesky, finish


def host_cpu() -> str:
    """Architecture and CPU model of the host (lscpu's model name when lscpu is present)."""
    import platform
    import subprocess
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{platform.machine()}, {model or platform.processor() or 'unknown model'}"


def cpu_baseline(P, n_s, steps=1):
    """Oracle NLL on the first n_s points (same m, m_v, d, kernel) -> evals/s of the
    full workload by linear scaling in n (the per-eval cost is O(n))."""
    from oracle import vif_oracle as O
    n = P.X.shape[0]
    Xs, ys = P.X[:n_s], P.y[:n_s]
    # neighbour sets for the timing sample: the m_v immediately preceding points
    # (the oracle's cost does not depend on which predecessors are chosen)
    N = -np.ones((n_s, P.mv), dtype=np.int64)
    for i in range(1, n_s):
        q = min(i, P.mv)
        N[i, :q] = np.arange(i - q, i)
    ts = []
    for _ in range(steps):
        t0 = time.time()
        O.VIF(Xs, P.Z, P.theta, N).nll(ys)
        ts.append(time.time() - t0)
    t = statistics.median(ts)
    return {"value": 1.0 / (t * n / n_s), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "host": host_cpu(),
            "sample": f"oracle NLL on the first {n_s} of {n} points (m={P.Z.shape[0]}, m_v={P.mv}, d=8), "
                      f"{t:.2f} s per sample eval, scaled by n/{n_s}"}


def small_configs_block(stream):
    """C2 (n = 100k, d = 2, Matern-5/2, m = 200, m_v = 30): NLL evals/s mixed and FP64 and their
    agreement; C1 (n = 2000, d = 2, Matern-3/2, m = 50, m_v = 10): latency of one NLL (both
    paths), one NLL with gradient and one prediction of 500 points.  Device-synchronised wall
    clock around the C-ABI calls, medians of repeated calls."""
    import torch
    from paper_2507_05064_gb300 import synth
    from paper_2507_05064_gb300 import vif as V

    def med_ms(fn, reps):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1000.0)
        return statistics.median(ts)

    out = {}
    P = synth.config2()
    c32 = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.MIXED, stream=stream.cuda_stream)
    c64 = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64, stream=stream.cuda_stream, neighbor_search=False)
    c64.set_neighbors(c32.neighbors())
    y = torch.from_numpy(P.y).cuda()
    t32 = med_ms(lambda: c32.nll(P.theta, y), 20)
    t64 = med_ms(lambda: c64.nll(P.theta, y), 5)
    a, b = c32.nll(P.theta, y), c64.nll(P.theta, y)
    out["c2"] = {"workload": "vif-nll-matern52-n100000-d2-m200-mv30", "mixed_evals_per_s": 1000.0 / t32,
                 "fp64_evals_per_s": 1000.0 / t64, "nll_mixed": a, "nll_fp64": b,
                 "rel_err_scale": abs(a - b) / max(abs(b), 0.5 * P.X.shape[0] * math.log(2 * math.pi))}
    c32.close()
    c64.close()
    P = synth.config1()
    c32 = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.MIXED, stream=stream.cuda_stream)
    c64 = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64, stream=stream.cuda_stream)
    y = P.y
    out["c1"] = {"workload": "matern32-n2000-d2-m50-mv10",
                 "nll_ms_mixed": med_ms(lambda: c32.nll(P.theta, y), 20),
                 "nll_ms_fp64": med_ms(lambda: c64.nll(P.theta, y), 20),
                 "nll_grad_ms_fp64": med_ms(lambda: c64.nll(P.theta, y, grad=True), 5),
                 "predict_500_ms_fp64": med_ms(lambda: c64.predict(P.theta, y, P.Xp), 10),
                 "timing": "host y and outputs, synchronised wall clock, median"}
    c32.close()
    c64.close()
    return out


def batch_block(args, stream):
    """Many independent problems (C5 recipe: n log-uniform in [2e3, 5e4], d in {2, 5},
    m in [64, 256], m_v in [10, 40]) likelihoods per CUDA graph replay, mixed path."""
    import torch
    from paper_2507_05064_gb300 import synth
    from paper_2507_05064_gb300 import vif as V
    t0 = time.time()
    probs = synth.config5(nprob=args.batch)
    gen_s = time.time() - t0
    t0 = time.time()
    ctxs = [V.Context(P.X, P.Z, P.mv, P.theta, precision=V.MIXED, stream=stream.cuda_stream) for P in probs]
    ys = [torch.from_numpy(P.y).cuda() for P in probs]
    torch.cuda.synchronize()
    build_s = time.time() - t0
    B = V.Batch(ctxs, [P.theta for P in probs], ys, stream=stream.cuda_stream)
    for _ in range(3):
        B.run()
    reps = 10
    t0 = time.perf_counter()
    for _ in range(reps):
        B.run()
    ms = (time.perf_counter() - t0) * 1000.0 / reps
    info = B.info()
    modes = {0: "per-problem launches", 1: "one persistent launch per bucket",
             2: "one flat launch per bucket (job records in the parameter bank)"}
    # the factor stage's other forms at the chosen branch count, for the record
    alt = {}
    if info["factor_buckets"] > 0:
        for mode in (0, 1, 2):
            if mode == info["batched_factor"]:
                continue
            B.set_shape(info["branches"], info["split_div"], mode)
            B.run()
            t1 = time.perf_counter()
            for _ in range(reps):
                B.run()
            alt[modes[mode]] = (time.perf_counter() - t1) * 1000.0 / reps
    npts = int(sum(P.X.shape[0] for P in probs))
    B.close()
    for c in ctxs:
        c.close()
    return {"workload": f"c5-{args.batch}-problems", "problems": args.batch, "points": npts,
            "ms_per_replay": ms, "problems_per_s": args.batch * 1000.0 / ms, "points_per_s": npts * 1000.0 / ms,
            "branches": info["branches"], "split_div": info["split_div"],
            "factor_stage": modes[info["batched_factor"]], "factor_buckets": info["factor_buckets"],
            "ms_per_replay_other_factor_forms": alt, "generate_s": gen_s,
            "build_s": build_s, "timing": "wall clock around vif_batch_run (graph replay + result read-back)"}


def laplace_block(args, stream):
    """Bernoulli-logit Laplace mode at n = 2e5 (Matern-3/2, range 0.05, m = 200, m_v = 20):
    Newton + PCG to relative residual 1e-6 with the plain VIFDU preconditioner."""
    import torch
    from paper_2507_05064_gb300 import synth
    from paper_2507_05064_gb300 import vif as V
    P = synth.config4(n=args.laplace_n)
    t0 = time.time()
    ctx = V.Context(P.X, P.Z, P.mv, P.theta, precision=V.FP64, likelihood=V.BERNOULLI_LOGIT,
                    stream=stream.cuda_stream)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    y = torch.from_numpy(P.y).cuda()
    ctx.laplace_mode(P.theta, y, rel_tol=1e-6)          # warm-up
    t0 = time.perf_counter()
    b_plain, st = ctx.laplace_mode(P.theta, y, rel_tol=1e-6)
    wall = time.perf_counter() - t0
    out = {"workload": f"laplace-bernoulli-matern32-n{P.X.shape[0]}-d2-m{P.Z.shape[0]}-mv{P.mv}",
           "rel_tol": 1e-6, "neighbor_build_s": build_s,
           "plain": {"precond": "VIFDU", "newton_iters": st["newton_iters"],
                     "pcg_iters_total": st["pcg_iters_total"], "ms_pcg": st["ms_pcg"],
                     "ms_total_device": st["ms_total"], "wall_s": wall, "objective": st["objective"]}}
    # the VIF-Laplace likelihood with the SLQ log-determinant (Eq. slq_v1): l = 50 probes (the
    # paper's default).  CG tolerance 1e-3 for VIFDU: at the paper's 0.01 its CG stops after ~5
    # Lanczos steps and the quadrature over-estimates this log-determinant by ~15% (measured on this
    # workload: 3857 at 1e-2, 3340 at 1e-3, 3333 at 1e-4 and 1e-6); FITC below is converged at 0.01.
    nprobe, slq_tol, fitc_tol = 50, 1e-3, 1e-2
    eps = synth.slq_normals(nprobe, P.Z.shape[0], P.X.shape[0])
    t0 = time.perf_counter()
    nll, sl = ctx.laplace_nll(P.theta, y, eps, slq_tol=slq_tol, rel_tol=1e-6)
    wall_slq = time.perf_counter() - t0
    out["slq"] = {"probes": nprobe, "cg_tol": slq_tol, "nll": nll, "logdet": sl["logdet"],
                  "logdet_exact_norm": sl["logdet_exact_norm"], "slq_term": sl["slq_term"],
                  "logdet_precond": sl["logdet_precond"], "pcg_iters_slq": sl["pcg_iters_slq"],
                  "ms_slq": sl["ms_slq"], "ms_per_probe": sl["ms_slq"] / nprobe, "ms_mode": sl["ms_mode"],
                  "wall_s": wall_slq,
                  "q_std_over_mean": float(np.std(sl["q"]) / max(abs(np.mean(sl["q"])), 1e-300))}
    # its gradient in (sigma1^2, lambda) by stochastic trace estimation with the same 50 probes and the
    # preconditioner control variate (Sec. 4.1, App. B, App. D); standard errors of the plain and the
    # control-variate trace estimates from the per-probe terms.  The traces reuse the probes' CG
    # solutions, which the gradient needs tighter than the log-determinant does: at the FITC form's
    # delta = 0.01 the two forms' gradients differed by 30-40 %, so both run at 1e-4 here.
    grad_tol = 1e-4
    t0 = time.perf_counter()
    nll_g, grad, sg = ctx.laplace_nll_grad(P.theta, y, eps, slq_tol=grad_tol, rel_tol=1e-6)
    wall_g = time.perf_counter() - t0
    pt, tr = sg["probe_terms"], sg["trace"]
    se_plain = pt[:, :, 0].std(axis=0, ddof=1) / np.sqrt(nprobe)
    se_cv = (pt[:, :, 0] - tr[None, :, 1] * pt[:, :, 1]).std(axis=0, ddof=1) / np.sqrt(nprobe)
    out["grad"] = {"params": ["sigma1^2", "lambda"], "cg_tol": grad_tol, "grad": grad.tolist(), "nll": nll_g,
                   "wall_s": wall_g,
                   "ms_after_nll": sg["ms_grad"], "pcg_iters_v": sg["pcg_iters_v"],
                   "trace_plain": tr[:, 0].tolist(), "c_opt": tr[:, 1].tolist(), "tau": tr[:, 2].tolist(),
                   "trace_cv": tr[:, 3].tolist(), "se_plain": se_plain.tolist(), "se_cv": se_cv.tolist(),
                   "wall_ratio_nll_grad_over_nll": wall_g / wall_slq}
    # the same with the FITC preconditioner (App. E.2, systems in the form of Eq. pcls2, Eq. slq_v2)
    ctx.laplace_mode(P.theta, y, rel_tol=1e-6, precond=V.PRECOND_FITC)          # warm-up
    t0 = time.perf_counter()
    b_f, sf = ctx.laplace_mode(P.theta, y, rel_tol=1e-6, precond=V.PRECOND_FITC)
    wall_f = time.perf_counter() - t0
    nll_f, slf = ctx.laplace_nll(P.theta, y, eps, slq_tol=fitc_tol, rel_tol=1e-6, precond=V.PRECOND_FITC)
    out["fitc"] = {"precond": "FITC (k = m, the VIF inducing points)", "newton_iters": sf["newton_iters"],
                   "pcg_iters_total": sf["pcg_iters_total"], "ms_pcg": sf["ms_pcg"],
                   "ms_total_device": sf["ms_total"], "wall_s": wall_f, "objective": sf["objective"],
                   "mode_rel_diff_vs_vifdu": float(np.linalg.norm(b_f - b_plain) / np.linalg.norm(b_plain)),
                   "slq": {"cg_tol": fitc_tol, "nll": nll_f, "logdet": slf["logdet"],
                           "logdet_exact_norm": slf["logdet_exact_norm"],
                           "pcg_iters_slq": slf["pcg_iters_slq"], "ms_slq": slf["ms_slq"],
                           "ms_per_probe": slf["ms_slq"] / nprobe}}
    # the gradient in the FITC form (Eq. pcls2 / slq_v2, App. D second form), same normals
    t0 = time.perf_counter()
    nll_gf, grad_f, sgf = ctx.laplace_nll_grad(P.theta, y, eps, slq_tol=grad_tol, rel_tol=1e-6,
                                               precond=V.PRECOND_FITC)
    wall_gf = time.perf_counter() - t0
    ptf, trf = sgf["probe_terms"], sgf["trace"]
    out["fitc"]["grad"] = {
        "cg_tol": grad_tol, "grad": grad_f.tolist(), "nll": nll_gf, "wall_s": wall_gf, "ms_after_nll": sgf["ms_grad"],
        "diff_vs_vifdu_form": (grad_f - grad).tolist(),
        "pcg_iters_v": sgf["pcg_iters_v"], "trace_cv": trf[:, 3].tolist(), "c_opt": trf[:, 1].tolist(),
        "se_plain": (ptf[:, :, 0].std(axis=0, ddof=1) / np.sqrt(nprobe)).tolist(),
        "se_cv": ((ptf[:, :, 0] - trf[None, :, 1] * ptf[:, :, 1]).std(axis=0, ddof=1) / np.sqrt(nprobe)).tolist()}
    # predictive means (Prop. 3.1) and SBPV variances (Alg. 1) at 1000 new points: 100 draws (the
    # paper's default), FITC solves at CG tolerance 0.01
    Xp = synth._rng(20250715).uniform(size=(1000, P.X.shape[1]))
    eps_p = synth.slq_normals(100, P.Z.shape[0], P.X.shape[0], seed=20250716)
    t0 = time.perf_counter()
    mu_p, var_p, sp = ctx.laplace_predict(P.theta, y, Xp, eps_p, cg_tol=1e-2, rel_tol=1e-6,
                                          precond=V.PRECOND_FITC)
    out["predict"] = {"n_pred": 1000, "samples": 100, "precond": "FITC", "cg_tol": 1e-2,
                      "wall_s": time.perf_counter() - t0, "ms_mode": sp["ms_total"],
                      "cg_iters_total": sp["pcg_iters_total"], "mean_abs_mean": float(np.abs(mu_p).mean()),
                      "mean_var": float(var_p.mean())}
    wpath = os.path.join(ROOT, "paper_2507_05064_gb300", "weights", "vifdu_mlp.npy")
    if os.path.exists(wpath):
        net = V.Network(params=np.load(wpath))
        ctx.laplace_mode(P.theta, y, rel_tol=1e-6, precond=1, mlp_weights=net)     # warm-up
        t0 = time.perf_counter()
        b_l, sl = ctx.laplace_mode(P.theta, y, rel_tol=1e-6, precond=1, mlp_weights=net)
        wall_l = time.perf_counter() - t0
        out["learned"] = {"precond": "VIFDU + learned diagonal correction", "newton_iters": sl["newton_iters"],
                          "pcg_iters_total": sl["pcg_iters_total"], "ms_pcg": sl["ms_pcg"],
                          "ms_total_device": sl["ms_total"], "wall_s": wall_l, "objective": sl["objective"],
                          "mode_rel_diff_vs_plain": float(np.linalg.norm(b_l - b_plain) / np.linalg.norm(b_plain))}
        out["pcg_time_ratio_learned_over_plain"] = sl["ms_pcg"] / st["ms_pcg"]
    ctx.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    P, _ = workload(args.n)
    cb = cpu_baseline(P, args.cpu_sample, steps=1)       # first warm-up step (also the calibration)
    vals = []
    for _ in range(max(args.warmup - 1, 0)):
        cpu_baseline(P, args.cpu_sample, steps=1)
    t0 = time.time()
    for _ in range(args.steps):
        vals.append(cpu_baseline(P, args.cpu_sample, steps=1)["value"])
    wall = time.time() - t0
    v = statistics.median(vals) if vals else cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(P, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "host": cb["host"], "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def run_vif(args, rank, world, dist):
    import torch
    from paper_2507_05064_gb300 import vif as V

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    P, gen_s = workload(args.n)
    th = P.theta
    t0 = time.time()
    ctx = V.Context(P.X, P.Z, P.mv, th, precision=V.MIXED, stream=stream.cuda_stream, stage_timing=True)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    rescored, fallback = ctx.knn_stats()
    N = ctx.neighbors()
    c64 = V.Context(P.X, P.Z, P.mv, th, precision=V.FP64, stream=stream.cuda_stream, neighbor_search=False)
    c64.set_neighbors(N)
    y_dev = torch.from_numpy(P.y).to(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.nll(th, y_dev)
    # the float32 factor stage's autotuned path (CUDA cores or tensor cores) and its timings
    factor_tuning = ctx.factor_tuning()
    stage_ms = {k: [] for k in V.STAGES}
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", 0)))
    barrier()
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    nll_mixed = None
    for _ in range(args.steps):
        nll_mixed = ctx.nll(th, y_dev)
        for k, v in ctx.stage_times().items():
            stage_ms[k].append(v)
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, dev)
    value = world * 1000.0 / ms

    # the analytic gradient in (sigma1^2, lambda_1..lambda_8, sigma^2) at this workload: the
    # mixed context forms it from one float64 pass (reverse mode), timed once after a warm-up
    grad_block = None
    if rank == 0 and world == 1:
        ctx.nll(th, y_dev, grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, g = ctx.nll(th, y_dev, grad=True)
        torch.cuda.synchronize()
        grad_block = {"params": ["sigma1^2"] + [f"lambda_{t + 1}" for t in range(P.X.shape[1])] + ["sigma^2"],
                      "grad": [float(x) for x in g], "ms_nll_and_grad": (time.perf_counter() - t0) * 1e3,
                      "precision": "float64 pass (reverse mode, App. A derivatives)"}

    # float64 GPU path on the same neighbour sets
    c64.nll(th, y_dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nll64 = None
    for _ in range(args.fp64_steps):
        nll64 = c64.nll(th, y_dev)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / max(args.fp64_steps, 1)
    # error of the mixed path against the float64 path, per output of the evaluation: the
    # likelihood and the factors it is built from (A_i and D_i of every point)
    A32, D32 = ctx.factors()
    A64, D64 = c64.factors()
    rD = (D32 - D64) / D64
    per_output = {"D_i": {"max_rel": float(np.abs(rD).max()), "mean_rel": float(rD.mean()),
                          "rms_rel": float(np.sqrt((rD ** 2).mean()))},
                  "A_i": {"max_abs": float(np.abs(A32 - A64).max()),
                          "rms_abs": float(np.sqrt(((A32 - A64) ** 2).mean()))},
                  "predictions": "a mixed context predicts through the float64 path (vif_predict): same values"}
    del A32, D32, A64, D64, rD

    # end to end through the C ABI with host buffers: y from pinned host memory, the
    # scalar back to the host, both inside the timed region
    y_pin = torch.from_numpy(P.y).pin_memory()
    y_host = y_pin.numpy()
    ctx.nll(th, y_host)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.nll(th, y_host)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0 / args.steps, dist, dev)

    if rank != 0:
        return
    med = {k: statistics.median(v) for k, v in stage_ms.items()}
    roof = roofline_block(P, med, ms, peaks(), factor_tuning.get("path", 1) if factor_tuning else 1)
    # the side blocks (Laplace rows, C1/C2, the oracle on the host cores) run at N = 1 only: at N > 1
    # the other GPUs would idle meanwhile and the CPU baseline is a single-GPU-run figure
    single = world == 1
    lap = None
    if not args.no_laplace and single:
        lap = laplace_block(args, stream)
    bat = batch_block(args, stream) if (args.batch > 0 and single) else None
    small = None if (args.no_small or not single) else small_configs_block(stream)
    cb = None
    if not args.no_cpu_baseline and single:
        cb = cpu_baseline(P, min(args.cpu_sample, P.X.shape[0]))
    have64 = nll64 is not None
    scale = max(abs(nll64), 0.5 * P.X.shape[0] * math.log(2 * math.pi)) if have64 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config_dict(P, world),
        "fp64_path": ({"value": world * 1000.0 / ms64, "unit": UNIT, "ms_per_step": ms64, "dtype": "f64"}
                      if have64 else None),
        "mixed_vs_fp64": ({"nll_mixed": nll_mixed, "nll_fp64": nll64,
                           "abs_err": abs(nll_mixed - nll64), "rel_err": abs(nll_mixed - nll64) / abs(nll64),
                           "rel_err_scale": abs(nll_mixed - nll64) / scale, "per_output": per_output}
                          if have64 else None),
        "speedup_mixed_over_fp64": ms64 / ms if have64 else None,
        "stage_ms": med,
        "neighbor_search": {"build_s": build_s, "queries_rescored": rescored, "queries_fallback": fallback},
        "factor_tuning": factor_tuning,
        "gradient": grad_block,
        "roofline": roof,
        "laplace": lap,
        "batch": bat,
        "small_configs": small,
        "cpu_baseline": cb,
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(P.y.nbytes) + 256, "d2h_bytes_per_step": 16 + 24},
        "gpu_launches": launches_per_eval(P.Z.shape[0]) * args.steps,
        "clocks": clocks,
        "generate_s": gen_s,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    c64.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.laplace_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        if rank == 0:
            print(json.dumps(laplace_block(args, torch.cuda.current_stream())), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    run_vif(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
