"""Runs a few tactile steps (forward, optionally reverse) of a named workload, for profilers.

    python -m paper_2604_20295_gb300.profile_step --workload hand --envs 4096 --precision bf16
    python -m paper_2604_20295_gb300.profile_step --workload flat16 --envs 1024 --backward
    python -m paper_2604_20295_gb300.profile_step --outputs count   # outputs of the bench step
    python -m paper_2604_20295_gb300.profile_step --envs 1024 --regress 3  # + taxel regressor

Workloads: ``hand`` (5 curved 16x32 fingertips + flat 32x64 palm per env), ``flat16`` (flat
16x16 pad pressed by a sphere), ``uneven`` (6 pads of 8x8 .. 64x64 nodes, 1-3 primitives).
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    import torch

    from . import build as B
    from . import etac as X
    from . import inputs as I

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="hand", choices=["hand", "flat16", "uneven"])
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--algo", default="batched", choices=["plain", "batched"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--backward", action="store_true")
    ap.add_argument("--outputs", default="all", choices=["all", "count"],
                    help="all: displacement, mask, penetration, active counts; count: "
                         "displacement and active counts (the benchmark's step)")
    ap.add_argument("--regress", type=int, default=0,
                    help="then run the taxel regressor (tensor-core path) this many times on "
                         "the last step's field")
    args = ap.parse_args()
    B.build()
    if args.workload == "hand":
        sc = I.hand_scene(args.envs, seed=2)
    elif args.workload == "flat16":
        sc = I.sphere_press_scene(args.envs, seed=7)
    else:
        sc = I.uneven_scene(args.envs, seed=5)
    sim = X.TactileSim(sc)
    sim.set_model(I.make_params(0), X.MODE_FULL,
                  X.PREC_BF16 if args.precision == "bf16" else X.PREC_FP32,
                  X.ALGO_BATCHED if args.algo == "batched" else X.ALGO_PLAIN)
    G = torch.as_tensor(np.random.default_rng(0).normal(size=(sc.total_nodes, 3)),
                        dtype=torch.float32).cuda()
    kw = {} if args.outputs == "all" else dict(want_mask=False, want_pen=False, want_count=True)
    for _ in range(args.steps):
        sim.step(**kw)
        if args.backward:
            sim.backward(G)
    extra = ""
    if args.regress:
        rp = torch.as_tensor(I.make_regressor_params(0)).cuda()
        for _ in range(args.regress):
            y, _ = sim.regress(rp, want_attn=False)
        extra = f" |taxels|={float(y.abs().sum()):.6e}"
    torch.cuda.synchronize()
    status = sim.poll_status()
    print(f"{args.workload} envs={args.envs} nodes={sc.total_nodes} status={status} "
          f"|disp|={float(sim.disp.abs().sum()):.6e}{extra}")
    sim.close()
    if status != 0:
        raise SystemExit(f"device status {status}")


if __name__ == "__main__":
    main()
