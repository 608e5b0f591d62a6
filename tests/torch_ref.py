"""Independent restatement of the ETac step in torch float64 on the CPU, used only to pin the
oracle.  It is written from the paper with library routines: ``torch.nn.functional.linear``,
``relu``, ``amax``, ``torch.cdist`` and autograd.  The outward SDF normal is obtained by
differentiating the signed distance with autograd (not by the hand-derived gradients and
Hessians of the oracle), and every reverse-mode quantity comes from autograd.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

from paper_2604_20295_gb300 import inputs as I


def _quat_mat(q):
    q = q / q.norm()
    x, y, z, w = q
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)]),
        torch.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)]),
        torch.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)])])


def _rodrigues(w):
    th = torch.sqrt((w * w).sum() + 1e-300)
    K = torch.stack([torch.stack([0 * w[0], -w[2], w[1]]),
                     torch.stack([w[2], 0 * w[0], -w[0]]),
                     torch.stack([-w[1], w[0], 0 * w[0]])])
    eye = torch.eye(3, dtype=w.dtype)
    # second-order expansion is exact enough at w = 0, where gradients are taken
    return eye + K + 0.5 * K @ K if float(th.detach()) < 1e-8 else \
        eye + torch.sin(th) / th * K + (1 - torch.cos(th)) / th ** 2 * K @ K


def sdf_inside_form(otype, dims, q):
    """Signed distance of a primitive, written in the form valid inside the object (where
    nodes are active) plus the exact outside form, evaluated with torch ops."""
    if otype == I.OBJ_SPHERE:
        return q.norm(dim=1) - dims[0]
    if otype == I.OBJ_BOX:
        d = q.abs() - torch.as_tensor(dims[:3], dtype=q.dtype)
        inside = (d <= 0).all(dim=1)
        out = torch.sqrt((d.clamp(min=0) ** 2).sum(1) + 1e-300)
        return torch.where(inside, d.max(dim=1).values, out)
    if otype == I.OBJ_CYLINDER:
        dr = torch.sqrt(q[:, 0] ** 2 + q[:, 1] ** 2) - dims[0]
        dz = q[:, 2].abs() - dims[1]
        inside = (dr <= 0) & (dz <= 0)
        out = torch.sqrt(dr.clamp(min=0) ** 2 + dz.clamp(min=0) ** 2 + 1e-300)
        return torch.where(inside, torch.maximum(dr, dz), out)
    if otype == I.OBJ_CAPSULE:
        cz = q[:, 2].clamp(-dims[1], dims[1])
        v = torch.stack([q[:, 0], q[:, 1], q[:, 2] - cz], 1)
        return v.norm(dim=1) - dims[0]
    raise ValueError(otype)


def network(P, Nrm, Uh, act, th):
    """Residual network Phi on one pad (Sec. III-A 2) -> per-node residual [n,3]."""
    X = torch.cat([P, Nrm, Uh * act[:, None]], 1)
    z1 = F.relu(F.linear(X, th["WE1"], th["bE1"]))
    f = F.relu(F.linear(z1, th["WE2"], th["bE2"]))
    g0 = f.amax(0)
    g = F.relu(F.linear(g0, th["WG1"], th["bG1"]))
    cat = torch.cat([f, g.expand(f.shape[0], -1)], 1)
    return F.linear(F.relu(F.linear(cat, th["WD1"], th["bD1"])), th["WD2"], th["bD2"])


def pad_output(P, Nrm, Uh, act, th, mode):
    """Eq. 4 on one pad: active nodes keep u_hat; passive nodes get Omega U_a + Phi_p."""
    if int(act.sum()) == 0:
        return torch.zeros_like(P)
    out = torch.zeros_like(P)
    if mode != 2:
        Om = torch.exp(-th["alpha"] * torch.cdist(P, P))
        out = out + Om[:, act] @ Uh[act]
    if mode != 1:
        out = out + network(P, Nrm, Uh, act.to(P.dtype), th)
    return torch.where(act[:, None], Uh, out)


def theta_tensors(theta, requires_grad=False):
    flat = torch.tensor(np.asarray(theta, np.float64), requires_grad=requires_grad)
    out = {}
    for k, (a, n, s) in I.param_slices().items():
        out[k] = flat[a] if not s else flat[a:a + n].reshape(s)
    return flat, out


def step(scene, theta, mode=0, mask=None, pose_leaves=False, uhat_override=None):
    """Whole step over a small scene.  Returns (disp [N,3], leaves dict).  With
    ``pose_leaves`` every object gets a translation increment and a left world-frame
    rotation increment (both zero) as autograd leaves; ``uhat_override`` makes u_hat a leaf
    (the mask must then be given)."""
    flat, th = theta_tensors(theta, requires_grad=True)
    leaves = {"params": flat}
    E, Pp, K = scene.num_envs, scene.pads_per_env, scene.max_objects
    dt = torch.zeros(E * K, 3, dtype=torch.float64, requires_grad=pose_leaves)
    dw = torch.zeros(E * K, 3, dtype=torch.float64, requires_grad=pose_leaves)
    leaves["dt"], leaves["dw"] = dt, dw
    offs = scene.node_offsets
    uo = None
    if uhat_override is not None:
        uo = torch.tensor(np.asarray(uhat_override, np.float64), requires_grad=True)
        leaves["uhat"] = uo
    outs = []
    for p in range(E * Pp):
        e = p // Pp
        t = scene.types[scene.pad_type[p]]
        P = torch.tensor(t.pos, dtype=torch.float64)
        Nrm = torch.tensor(t.nrm, dtype=torch.float64)
        pp = torch.tensor(scene.pad_pose.reshape(-1, 7)[p], dtype=torch.float64)
        Rp, tp = _quat_mat(pp[3:]), pp[:3]
        x = P @ Rp.T + tp
        a, b = offs[p], offs[p + 1]
        if uo is not None:
            act = torch.tensor(np.asarray(mask[a:b]) != 0)
            Uh = uo[a:b]
        else:
            best, bphi, bU = None, None, None
            for k in range(K):
                o = e * K + k
                ot = int(scene.obj_type[o])
                if ot == 0:
                    continue
                op = torch.tensor(scene.obj_pose.reshape(-1, 7)[o], dtype=torch.float64)
                Rk = _rodrigues(dw[o]) @ _quat_mat(op[3:])
                tk = op[:3] + dt[o]
                q = (x - tk) @ Rk                  # rows are R_k^T (x - t_k)
                dims = [float(v) for v in scene.obj_dims.reshape(-1, 3)[o]]
                qg = q if q.requires_grad else q.detach().requires_grad_(True)
                phi = sdf_inside_form(ot, dims, qg)
                grad = torch.autograd.grad(phi.sum(), qg, create_graph=True)[0]
                u_obj = -phi[:, None] * grad
                U = (u_obj @ Rk.T) @ Rp            # object -> world -> pad frame
                if best is None:
                    best, bphi, bU = torch.full((len(P),), k), phi, U
                else:
                    better = phi < bphi
                    bphi = torch.where(better, phi, bphi)
                    bU = torch.where(better[:, None], U, bU)
            if mask is not None:
                act = torch.tensor(np.asarray(mask[a:b]) != 0)
            else:
                act = (bphi < 0).detach()
            Uh = bU * act[:, None]
        outs.append(pad_output(P, Nrm, Uh, act, th, mode))
    return torch.cat(outs, 0), leaves
