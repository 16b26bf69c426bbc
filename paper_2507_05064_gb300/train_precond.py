"""Train the learned diagonal correction of the VIFDU preconditioner.

Training systems are the Newton iterates of Bernoulli-logit Laplace problems the
method itself generates: n = 20,000 points uniform on [0,1]^2, Matern-3/2 latent
GP (variance 1, range log-uniform in [0.03, 0.1]), m = 200 k-means++ inducing
points, m_v = 20; each problem contributes `newton` systems.  At every system the
network takes `steps` Adam steps on the Hutchinson estimate of
||P^{-1}(W + Sigma_dagger^{-1}) - I||_F^2 (vif_mlp_train).  The float32 parameters
are saved with numpy (VIF_MLP_NPARAM values in the packed order of include/vif.h).

    python -m paper_2507_05064_gb300.train_precond --systems 5000 --out weights.npy
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_training_problem(k: int, n: int):
    from paper_2507_05064_gb300 import synth
    rng = np.random.default_rng(777_000 + k)
    rho = float(math.exp(rng.uniform(math.log(0.03), math.log(0.1))))
    P = synth.make_problem(n, 2, 200, 20, "matern32", 1.0, rho, 0.0, 5_000_000 + k,
                           likelihood="bernoulli_logit", lloyd=2, rff=256)
    return P.X, P.y, P.Z, rho


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=5000)
    ap.add_argument("--n", type=int, default=20_000)
    ap.add_argument("--newton", type=int, default=5)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--probes", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "vifdu_mlp.npy"))
    args = ap.parse_args()
    nprob = (args.systems + args.newton - 1) // args.newton
    # the generator pool is started with spawn before any CUDA work in this process
    pool = mp.get_context("spawn").Pool(args.workers)
    jobs = [pool.apply_async(make_training_problem, (k, args.n)) for k in range(nprob)]

    from paper_2507_05064_gb300 import synth
    from paper_2507_05064_gb300 import vif as V
    net = V.Network(seed=args.seed)
    t0 = time.time()
    log = []
    systems = 0
    for k, job in enumerate(jobs):
        X, y, Z, rho = job.get()
        th = synth.Theta(1, 1.0, np.array([rho]), 0.0)
        ctx = V.Context(X, Z, 20, th, precision=V.FP64, likelihood=V.BERNOULLI_LOGIT)
        st = ctx.mlp_train(th, y, net, steps_per_system=args.steps, probes=args.probes,
                           max_newton=args.newton, lr=args.lr, seed=args.seed * 100_003 + k)
        ctx.close()
        systems += st["systems"]
        log.append([k, rho, st["loss_first"], st["loss_last"]])
        if k % 50 == 0:
            print(f"problem {k} systems {systems} loss {st['loss_first']:.4f} -> {st['loss_last']:.4f} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    pool.close()
    params = net.params()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, params)
    summary = {"systems": systems, "problems": nprob, "n": args.n, "steps_per_system": args.steps,
               "probes": args.probes, "lr": args.lr, "seconds": time.time() - t0,
               "loss_first_mean_first50": float(np.mean([r[2] for r in log[:50]])),
               "loss_last_mean_last50": float(np.mean([r[3] for r in log[-50:]]))}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
