"""Calibration of the propagation model (ETac Sec. III-A, Eq. 5).

The paper fits alpha and the residual network by gradient descent on the error of passive-
node displacements against reference displacements.  ``fit`` runs that loop on the GPU:
forward and reverse mode through the C ABI (``etac_step_forward`` / ``etac_step_backward``),
Adam (torch.optim) on the flat parameter vector.  The loss is the mean squared error over
passive nodes (Eq. 5 writes the 2-norm; both have the same minimiser, and the norm is
returned as well).  Usage: ``python -m paper_2604_20295_gb300.fit targets.npz`` runs the
1,024-env calibration against stored target displacements.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import etac as X
from . import inputs as I


def fit(scene, theta0, target_disp, iters: int = 200, lr: float = 1e-3, betas=(0.9, 0.999),
        mode: int = X.MODE_FULL, algo: int = X.ALGO_BATCHED, device: str = "cuda",
        log_every: int = 0) -> dict:
    import torch

    sim = X.TactileSim(scene, device=device)
    try:
        sim.set_model(theta0, mode, X.PREC_FP32, algo)
        params = torch.nn.Parameter(torch.as_tensor(np.asarray(theta0, np.float32), device=sim.device))
        opt = torch.optim.Adam([params], lr=lr, betas=betas)
        target = torch.as_tensor(np.asarray(target_disp, np.float32), device=sim.device)
        losses, norms, alphas = [], [], []
        t0 = time.perf_counter()
        for it in range(iters + 1):
            sim.set_model(params.detach(), mode, X.PREC_FP32, algo)
            disp = sim.step()
            passive = sim.mask == 0     # Eq. 5 scores passive nodes (contact set is fixed)
            npas = max(int(passive.sum()), 1)
            diff = (disp - target) * passive[:, None]
            loss = float((diff * diff).sum()) / (3 * npas)
            losses.append(loss)
            norms.append(float(diff.norm()))
            alphas.append(float(params.detach()[0]))
            if log_every and it % log_every == 0:
                print(f"iter {it:4d} loss {loss:.6e} |dU| {norms[-1]:.4e} alpha {alphas[-1]:.5f}")
            if it == iters:
                break
            grads = sim.backward(diff * (2.0 / (3 * npas)), want=("params",))
            opt.zero_grad()
            params.grad = grads["params"]
            opt.step()
            with torch.no_grad():
                params[0].clamp_(min=1e-3)   # alpha > 0
        torch.cuda.synchronize()
        return {"loss": losses, "norm": norms, "alpha": alphas,
                "params": params.detach().cpu().numpy(), "seconds": time.perf_counter() - t0}
    finally:
        sim.close()


def passive_rms(scene, theta, target_disp, mode: int = X.MODE_FULL, algo: int = X.ALGO_BATCHED,
                device: str = "cuda") -> float:
    """Root-mean-square error (mm) of the passive nodes' displacements of the model `theta`
    against `target_disp` on `scene` (the quantity Eq. 5 fits), one FP32 forward step."""
    import torch

    sim = X.TactileSim(scene, device=device)
    try:
        sim.set_model(theta, mode, X.PREC_FP32, algo)
        disp = sim.step()
        passive = sim.mask == 0
        target = torch.as_tensor(np.asarray(target_disp, np.float32), device=sim.device)
        diff = (disp - target) * passive[:, None]
        n = max(int(passive.sum()), 1)
        return float(torch.sqrt((diff * diff).sum() / (3 * n)))
    finally:
        sim.close()


def main():
    ap = argparse.ArgumentParser(description="Eq. 5 calibration to stored target displacements")
    ap.add_argument("targets", help=".npz with 'disp' [N, 3] for sphere_press_scene(envs, seed=7)")
    ap.add_argument("--envs", type=int, default=1024)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    scene = I.sphere_press_scene(args.envs, seed=7)
    target = np.load(args.targets)["disp"]
    if target.shape != (scene.total_nodes, 3):
        raise SystemExit(f"targets have shape {target.shape}, the scene has {scene.total_nodes} nodes")
    th0 = I.make_params(args.seed)
    h = fit(scene, th0, target, iters=args.iters, lr=args.lr)
    print(json.dumps({"envs": args.envs, "iters": args.iters, "loss_first": h["loss"][0],
                      "loss_last": h["loss"][-1], "norm_first": h["norm"][0],
                      "norm_last": h["norm"][-1], "alpha_start": float(th0[0]),
                      "alpha_end": h["alpha"][-1], "seconds": h["seconds"]}))


if __name__ == "__main__":
    main()
