"""Times the GPU signed-distance query against a closed triangle mesh on the nodes of the
hand workload pressed into a rock mesh, and prints one JSON line.

    python -m paper_2604_20295_gb300.profile_mesh --envs 4096 --reps 20

Workload: ``inputs.mesh_scene`` with one shared 1,280-triangle rock (4,096 envs x 6 pads,
18,874,368 nodes).  The nodes' object-frame positions are formed once on the GPU (torch),
then ``etac_mesh_sdf_query`` runs over all of them ``reps`` times, timed with CUDA events on
the launching stream after ``warmup`` untimed runs.  The 226 MB input and 302 MB output are
larger than L2, so every run reads and writes HBM.  Reported: milliseconds per query, points
per second, the share of points in listed cells, listed triangles visited per point, HBM
bytes per second (12 B in, 16 B out per point) against the measured copy bandwidth, and the
share of points inside the mesh.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np


def _rot(q):
    import torch
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    x, y, z, w = q.unbind(-1)
    return torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                        2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                        2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
                       -1).reshape(*q.shape[:-1], 3, 3)


def main():
    import torch

    from . import build as B
    from . import etac as X
    from . import inputs as I

    ap = argparse.ArgumentParser()
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--grid", type=int, default=32)
    args = ap.parse_args()
    B.build()
    sc = I.mesh_scene(args.envs, seed=3, num_meshes=1)
    mesh = sc.meshes[0]
    dev = torch.device("cuda")
    # object-frame position of every node: q = R_o^T (R_p p + t_p - t_o)
    offs = sc.node_offsets
    type_of_node = np.repeat(sc.pad_type, np.diff(offs))
    local = np.concatenate([sc.types[t].pos for t in sc.pad_type]).astype(np.float32)
    pad_of_node = np.repeat(np.arange(len(sc.pad_type)), np.diff(offs))
    env_of_node = pad_of_node // sc.pads_per_env
    pp = torch.as_tensor(sc.pad_pose.reshape(-1, 7), device=dev)
    op = torch.as_tensor(sc.obj_pose.reshape(-1, 7), device=dev)
    pn = torch.as_tensor(pad_of_node, device=dev)
    en = torch.as_tensor(env_of_node, device=dev)
    p = torch.as_tensor(local, device=dev)
    world = torch.einsum("nij,nj->ni", _rot(pp[:, 3:])[pn], p) + pp[pn, :3]
    q = torch.einsum("nji,nj->ni", _rot(op[:, 3:])[en], world - op[en, :3]).contiguous()
    del world, p, pn, en
    n = q.shape[0]
    assert n == sc.total_nodes and type_of_node.size == n

    sdf = X.MeshSDF(mesh.verts, mesh.tris, args.grid)
    acc = X.mesh_accel(mesh.verts, mesh.tris, args.grid)
    phi = torch.empty(n, dtype=torch.float32, device=dev)
    grad = torch.empty(n, 3, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    run = lambda: X.etac_mesh_sdf_query(sdf.handle, n, q.data_ptr(), phi.data_ptr(),
                                        grad.data_ptr(), stream.cuda_stream)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.reps):
        run()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.reps

    # listed triangles per point, from the grid the query reads (float32 cell lookup)
    qh = q.cpu().numpy()
    rel = (qh - acc["origin"]) / np.float32(acc["cell"])
    dims = np.array(acc["dims"])
    ok = np.all((rel >= 0) & (rel < dims), axis=1)
    ijk = np.minimum(np.floor(np.where(ok[:, None], rel, 0)).astype(np.int64), dims - 1)
    cell = (ijk[:, 2] * dims[1] + ijk[:, 1]) * dims[0] + ijk[:, 0]
    count = np.where(ok, np.diff(acc["cell_start"])[cell], 0)
    ph = phi.cpu().numpy()
    sdf.close()
    peaks_path = os.path.join(B.ROOT, "MEASURED_PEAKS.json")
    hbm = None
    if os.path.exists(peaks_path):
        try:
            hbm = float(json.load(open(peaks_path)).get("hbm_gbs"))
        except (ValueError, TypeError):
            hbm = None
    gbs = 28.0 * n / (ms * 1e-3) / 1e9
    print(json.dumps(dict(
        kernel="mesh_sdf_kernel", workload=f"hand-mesh {args.envs} envs, rock {len(mesh.tris)} tris, grid {args.grid}",
        points=n, ms=round(ms, 4), points_per_s=n / (ms * 1e-3),
        listed_frac=float(np.mean(count > 0)), cand_per_point=float(count.mean()),
        cand_per_listed_point=float(count[count > 0].mean()) if np.any(count > 0) else 0.0,
        cand_visits_per_s=float(count.sum()) / (ms * 1e-3),
        hbm_gbs=gbs, hbm_peak_gbs=hbm, hbm_frac=(gbs / hbm) if hbm else None,
        inside_frac=float(np.mean(ph < 0)))))


if __name__ == "__main__":
    main()
