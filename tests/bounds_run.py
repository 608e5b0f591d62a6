"""Child process of tests/test_gpu_bounds.py: runs every GPU path once on small seeded scenes
(each forward algorithm and precision in every mode, mode B, mesh objects, the reverse mode of
both algorithms, the regressor in both precisions) with the library ETAC_LIBRARY names, and
saves all outputs and the device status word after each call to the .npz file given."""
import sys

import numpy as np
import torch

from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I


def main(path):
    out = {}

    def keep(name, sim, **tensors):
        torch.cuda.synchronize()
        out[name + ":status"] = np.array(sim.poll_status())
        for k, t in tensors.items():
            out[f"{name}:{k}"] = t.detach().cpu().numpy().copy()

    theta = I.make_params(0)
    sc = I.hand_scene(24, seed=4)
    G = torch.as_tensor(np.random.default_rng(1).normal(size=(sc.total_nodes, 3)),
                        dtype=torch.float32).cuda()
    for algo, prec in ((X.ALGO_PLAIN, X.PREC_FP32), (X.ALGO_BATCHED, X.PREC_FP32),
                       (X.ALGO_BATCHED, X.PREC_BF16)):
        for mode in (X.MODE_FULL, X.MODE_LINEAR_ONLY, X.MODE_RESIDUAL_ONLY,
                     X.MODE_PENETRATION_ONLY):
            sim = X.TactileSim(sc)
            try:
                sim.set_model(theta, mode, prec, algo)
                sim.step()
                tag = f"hand:{algo}:{prec}:{mode}"
                keep(tag, sim, disp=sim.disp, mask=sim.mask, pen=sim.pen, count=sim.count)
                if mode == X.MODE_FULL:
                    g = sim.backward(G)
                    keep(tag + ":bwd", sim, **{k: v for k, v in g.items() if torch.is_tensor(v)})
                    # mode B: the forward contact set and u_hat supplied by the caller
                    uh = torch.where(sim.mask.bool()[:, None], sim.disp, torch.zeros_like(sim.disp))
                    sim.step(uhat_in=uh.contiguous(), mask_in=sim.mask.clone())
                    keep(tag + ":modeB", sim, disp=sim.disp)
            finally:
                sim.close()
    un = I.uneven_scene(8, seed=6)
    sim = X.TactileSim(un)
    try:
        sim.set_model(theta, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        sim.step()
        keep("uneven:bf16", sim, disp=sim.disp, mask=sim.mask)
    finally:
        sim.close()
    ms = I.mesh_scene(6, seed=5)
    sim = X.TactileSim(ms)
    try:
        sim.set_model(theta, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        sim.set_meshes()
        sim.step()
        keep("mesh:bf16", sim, disp=sim.disp, mask=sim.mask)
    finally:
        sim.close()
    rp = I.make_regressor_params(2)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(theta, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        sim.step()
        for prec in (X.PREC_BF16, X.PREC_FP32):
            y, a = sim.regress(rp, precision=prec)
            keep(f"regress:{prec}", sim, taxels=y, attn=a)
    finally:
        sim.close()
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
