"""Benchmark of the ETac tactile step on GB300: node-steps/s over 4,096 environments.

Workload (default): 4,096 environments x (5 curved 16x32 fingertip pads + one flat 32x64 palm
pad) = 18,874,368 surface nodes per step, one seeded primitive per environment (sphere, box,
cylinder or capsule), penetration 0-3 mm, seeded propagation-model parameters (seed 0).  One
step = contact detection + Eq. 1 propagation + residual network + Eq. 4 for every node.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the host
cores instead (bounded env sample per step).  Under torchrun each rank runs an independent
replica on its own GPU (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_20295_gb300 import inputs as I  # noqa: E402

METRIC = "tactile node-steps/sec at 4096 envs (BF16 batched vs FP32 plain) at stated err; bwd/fwd"
UNIT = "node-steps/s"
H = 64


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def max_over_ranks(x, pg, device):
    """The largest of every rank's x (the job's time is its slowest rank's), via the process
    group `pg` (torch.distributed, or None for one process); float64 tensor on `device`."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t)


def job_rate(nodes_per_rank_step, steps, world, seconds):
    """Whole-job node-steps/s: every rank runs its own replica of the workload (weak scaling),
    so the job processes nodes x steps x world in the slowest rank's time."""
    return nodes_per_rank_step * steps * world / seconds


def algorithmic_work(scene, counts):
    """FLOPs and bytes the method itself requires per step (implementation overheads such as
    recomputation or padding are not counted).  counts = active nodes per pad."""
    n = scene.pad_nodes.astype(np.float64)
    m = counts.astype(np.float64)
    passive = np.where(m > 0, n - m, 0.0)
    active = np.where(m > 0, m, 0.0)
    pairs = float((passive * active).sum())
    enc = 2.0 * (NIN_H + H * H)            # E1 + E2 per node
    dec = 2.0 * (H * H + 3 * H)            # D1 (per-node half) + D2 per passive node
    literal = float((n * (m > 0)).sum()) * enc + float(passive.sum()) * dec + 6.0 * pairs
    bytes_out = 12.0 * float(n.sum())      # displacement, float32 x3
    return dict(pairs=pairs, literal_flops=literal, bytes_out=bytes_out,
                active=float(active.sum()), passive=float(passive.sum()))


NIN_H = 9 * H

# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of the kernel
# named, valid only for the source hash recorded with it (null once the kernel changes)
TRAFFIC = {
    # hand workload, 4,096 envs, one pass of --metrics
    # gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum (profile_step --outputs
    # count: the bench step's outputs; --backward for the reverse stages); per stage where a
    # stage is several kernels
    "front_contact_kernel": {"file": "paper_2604_20295_gb300/csrc/front.cu",
                             "sha": "56c1d146a20d5381", "bytes": 42.75e6 + 59.40e6},
    "front_global_kernel": {"file": "paper_2604_20295_gb300/csrc/front.cu",
                            "sha": "56c1d146a20d5381", "bytes": 6.55e6},
    "prop_gemm_kernel": {"file": "paper_2604_20295_gb300/csrc/prop_gemm.cu",
                         "sha": "59f10d54de88bcd0", "bytes": 136.38e6 + 127.49e6},
    "prop_gemm_kernel<bwd_u>": {"file": "paper_2604_20295_gb300/csrc/prop_gemm.cu",
                                "sha": "59f10d54de88bcd0", "bytes": 332.76e6 + 44.29e6},
    "prop_gemm_kernel<bwd_alpha>": {"file": "paper_2604_20295_gb300/csrc/prop_gemm.cu",
                                    "sha": "59f10d54de88bcd0", "bytes": 331.07e6 + 0.16e6},
    "bwd_pad_kernel": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",
                       "sha": "7c174cf342576933", "bytes": 246.44e6 + 325.39e6},
    "bwd_global_kernel": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",
                          "sha": "7c174cf342576933", "bytes": 8.81e6 + 0.01e6},
    "bwd_decoder_kernel": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",
                           "sha": "7c174cf342576933", "bytes": 238.84e6 + 65.62e6},
    "bwd_reduce_a3_kernel": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",
                             "sha": "7c174cf342576933", "bytes": 75.51e6 + 0.02e6},
    "bwd_padrev_kernel": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",   # + padmlp
                          "sha": "7c174cf342576933", "bytes": 52.27e6 + 2.45e6 + 34.23e6 + 0.07e6},
    "bwd_padsum_kernel": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",
                          "sha": "7c174cf342576933", "bytes": 102.40e6 + 11.75e6},
    # bwd_fill_kernel + bwd_pose_kernel + bwd_reduce_params_kernel
    "bwd_pose_kernel(+param sums)": {"file": "paper_2604_20295_gb300/csrc/bwd_batched.cu",
                                     "sha": "7c174cf342576933",
                                     "bytes": 95.16e6 + 228.16e6 + 97.71e6 + 7.37e6 + 30.29e6},
}


# warp instructions per node of an issue-bound kernel (smsp__inst_executed.sum of one
# --set full capture, hand workload at 2,048 envs = 9,437,184 nodes), valid for the source hash
INSTR = {
    "front_contact_kernel": {"file": "paper_2604_20295_gb300/csrc/front.cu",
                             "sha": "56c1d146a20d5381", "per_node": 122214527 / 9437184},
}


def instr_per_node(name):
    """Recorded warp instructions per node of kernel `name`, or None once its source changed."""
    import hashlib
    rec = INSTR.get(name)
    if not rec:
        return None
    try:
        with open(os.path.join(ROOT, rec["file"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return rec["per_node"] if sha == rec["sha"] else None


def traffic_for(name):
    """Recorded DRAM bytes per launch of kernel `name`, or None when the kernel's source file
    no longer has the hash the capture was taken with."""
    import hashlib
    rec = TRAFFIC.get(name)
    if not rec:
        return None
    try:
        with open(os.path.join(ROOT, rec["file"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return rec["bytes"] if sha == rec["sha"] else None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen([exe, f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                      "-i", str(self.index), "-lms", "200"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def parse_cpulist(text):
    """The CPU set of a Linux cpulist string ("0-3,8,10-11")."""
    cpus = set()
    for part in text.strip().split(","):
        part = part.strip()
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(torch, dev):
    """The CPUs of the GPU's own NUMA node that this process may use (Linux sysfs
    local_cpulist of the GPU's PCI function), or None where the system does not say."""
    try:
        p = torch.cuda.get_device_properties(dev)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            cpus = parse_cpulist(f.read())
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


def oracle_rate(scene, theta, sample_envs, nthreads=0):
    """Times the FP64 oracle (as it stands) on a bounded env sample; node-steps/s."""
    import oracle
    sub = scene.subset(sample_envs)
    t0 = time.perf_counter()
    oracle.forward(sub, theta, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return sub.total_nodes / dt, dt, sub.total_nodes


def oracle_single_core(scene, theta, sample_envs):
    """The oracle's single-thread rate on a small env sample.  OpenMP keeps the thread count
    set for a call, so the all-core count is put back afterwards (one env, untimed)."""
    rate, dt, nn = oracle_rate(scene, theta, sample_envs, nthreads=1)
    oracle_rate(scene, theta, sample_envs[:1], nthreads=cpu_cores())
    return rate, dt, nn


def run_reference(args, scene, theta, rank, world):
    if rank != 0:
        return
    rng = np.random.default_rng(123)
    times, nodes = [], 0
    for it in range(args.warmup + args.steps):
        envs = rng.choice(scene.num_envs, args.ref_envs, replace=False)
        rate, dt, nn = oracle_rate(scene, theta, envs)
        if it >= args.warmup:
            times.append(dt)
            nodes += nn
    value = nodes / sum(times)
    cores = cpu_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, scene),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_envs} random envs ({args.ref_envs * 4608} nodes) "
                                       "of the workload per step, FP64 C oracle, OpenMP over pads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, scene):
    return {"workload": f"hand-{scene.num_envs}env-5tip16x32r8-palm32x64",
            "envs": scene.num_envs, "pads_per_env": scene.pads_per_env,
            "nodes_per_step": scene.total_nodes, "algo": args.algo, "precision": args.precision,
            "l2": "flushed between timed steps (256 MiB write)", "params_seed": 0,
            "scene_seed": args.seed}


def timed_steps(sim, steps, stream, flush, torch, step_kw):
    """K steps, L2 flushed between them outside the events; returns per-step ms."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        sim.step(**step_kw)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def executed_gemm_flops(scene):
    """Dense FLOPs the tensor-core propagation executes: 2 n_t^2 * 3 per instance."""
    n = scene.pad_nodes.astype(np.float64)
    return float((2.0 * n * n * 3.0).sum())


def bwd_rooflines(ktimes, scene, work, peaks, nsm):
    """Per-stage time and roofline of the staged reverse mode.  Algorithmic work per stage (what
    the reverse of the method needs, not the implementation's recomputation or split products):
      pad stage   -- read dL/dU (12 B per node), write the passive gradient as the propagation
                     reverse's operand (BF16, 6 B per node) and u_hat / phi of active nodes
                     (16 B): HBM;
      decoder     -- per passive node dz = D2^T g (384 FLOP), dD2 (384 FLOP), the S and A3
                     sums (128 FLOP): FP32 ALU; its A3 sums read the partials (4 B per type
                     node and channel per group; counted once per node: HBM);
      pad reverse -- per pad D1_g^T S and G1^T dag (16.4 kFLOP) and at most 64 routed nodes'
                     E2 / E1 reverse (2 x (64 + 576 + 192) FLOP per routed channel): FP32 ALU;
      pad sums    -- per pad the outer products S g^T, dag g0^T (16.4 kFLOP) and dA2 h1^T
                     (8.2 kFLOP): FP32 ALU;
      GEMMs       -- 6 FLOP per (passive, active) pair each (dL/du_hat and d alpha): tensor;
      outputs     -- read the propagated dL/du_hat and write dL/du_hat, dL/dpen (28 B per
                     node): HBM;
      A3 sums     -- read the per-64-instance partials of each type node and channel once and
                     write their sums: HBM.
    FP32 ALU peak = SMs x 128 lanes x 2 FLOP x max SM clock."""
    nodes = float(scene.total_nodes)
    npads = float(scene.num_envs * scene.pads_per_env)
    alu = nsm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    # the A3 sums (decoder reverse, per type node and channel) are reduced from one partial per
    # group of 64 instances of the type: read every partial once, write the sums (HBM bytes of
    # the implementation's reduction; the method itself only needs the sums)
    inst = np.bincount(np.asarray(scene.pad_type), minlength=len(scene.types))
    tn = np.asarray(scene.type_num_nodes, np.float64)
    a3_bytes = float((4.0 * H * tn * (np.ceil(inst / 64.0) + 1.0)).sum())
    spec = {"bwd_pad_kernel": ("hbm", 18.0 * nodes + 16.0 * work["active"]),
            "bwd_global_kernel": ("alu", npads * 2.0 * 2 * H * H),
            "bwd_decoder_kernel": ("alu", 896.0 * work["passive"]),
            "bwd_reduce_a3_kernel": ("hbm", a3_bytes),
            "bwd_padrev_kernel": ("alu", npads * (2.0 * 2 * H * H + H * 2.0 * (64 + 576 + 192))),
            "bwd_padsum_kernel": ("alu", npads * (2.0 * 2 * H * H + 2.0 * H * H)),
            "prop_gemm_kernel<bwd_u>": ("tensor", 6.0 * work["pairs"]),
            "prop_gemm_kernel<bwd_alpha>": ("tensor", 6.0 * work["pairs"]),
            "bwd_pose_kernel(+param sums)": ("hbm", 28.0 * nodes)}
    out = {}
    for name, (launches, ms) in ktimes.items():
        t = ms / max(launches, 1) / 1e3
        ent = {"ms": t * 1e3}
        if name in spec and t > 0:
            bound, w = spec[name]
            ent["traffic"] = traffic_for(name) if scene.num_envs == 4096 else None
            if bound == "hbm":
                a, p, u = w / t / 1e9, peaks["hbm_gbs"], "GB/s"
            elif bound == "tensor":
                a, p, u = w / t / 1e12, peaks["bf16_tflops"], "TFLOP/s"
            else:
                a, p, u = w / t / 1e12, alu, "TFLOP/s"
            ent.update(bound=bound, achieved=a, peak=p, unit=u, frac=a / p)
        out[name] = ent
    return out


def _stats(got, ref_disp, mask_got, mask_ref):
    d = np.linalg.norm(got.astype(np.float64) - ref_disp, axis=1)
    return {"max_abs_mm": float(d.max()), "rms_mm": float(np.sqrt((d ** 2).mean())),
            "mask_mismatch_nodes": int((mask_got != mask_ref).sum())}


def config_c3(X, I, torch, dev, stream, flush, theta, with_oracle):
    """The single-pad sphere-press workload (100 seeded steps, flat 16x16 pad) in FP32 plain and
    with the BF16 tensor-core propagation: time per launch of all 100 steps as 100 problems,
    the one-step latency, and the error of each against the FP64 oracle."""
    sc = I.sphere_press_scene(100, seed=0)
    out = {"workload": "sphere-press 16x16 flat pad, 100 seeded steps as 100 problems per launch"}
    runs = {}
    for name, prec, algo in [("fp32_plain", X.PREC_FP32, X.ALGO_PLAIN),
                             ("bf16_batched", X.PREC_BF16, X.ALGO_BATCHED)]:
        sim = X.TactileSim(sc, device=dev)
        sim.set_model(theta, X.MODE_FULL, prec, algo)
        for _ in range(3):
            sim.step()
        ms = timed_steps(sim, 20, stream, flush, torch, {})
        sim.step()
        torch.cuda.synchronize()
        runs[name] = {"us_per_launch": 1e3 * sum(ms) / len(ms),
                      "disp": sim.disp.cpu().numpy(), "mask": sim.mask.cpu().numpy()}
        sim.close()
        one = X.TactileSim(sc.subset([0]), device=dev)
        one.set_model(theta, X.MODE_FULL, prec, algo)
        for _ in range(3):
            one.step()
        ms1 = timed_steps(one, 20, stream, flush, torch, {})
        runs[name]["us_one_step"] = 1e3 * sum(ms1) / len(ms1)
        one.close()
    out["fp32_plain_us_per_launch"] = runs["fp32_plain"]["us_per_launch"]
    out["bf16_us_per_launch"] = runs["bf16_batched"]["us_per_launch"]
    out["fp32_plain_us_one_step"] = runs["fp32_plain"]["us_one_step"]
    out["bf16_us_one_step"] = runs["bf16_batched"]["us_one_step"]
    out["throughput_ratio_bf16_over_fp32"] = (runs["fp32_plain"]["us_per_launch"] /
                                              runs["bf16_batched"]["us_per_launch"])
    if with_oracle:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.forward(sc, theta)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": sc.total_nodes / dt, "unit": UNIT, "cores": cpu_cores(),
                               "kind": "oracle", "us_per_step": 1e6 * dt / sc.num_envs,
                               "sample": f"all {sc.num_envs} steps ({sc.total_nodes} nodes), "
                                         f"FP64 forward, OpenMP over pads, {dt:.3f} s"}
        for name in runs:
            out[f"{name}_error"] = _stats(runs[name]["disp"], ref["disp"], runs[name]["mask"],
                                          ref["mask"])
    return out


def config_c4_fit(I, theta0, with_oracle):
    """Eq. 5 calibration over 1,024 envs of the single-pad layout: Adam, 200 iterations, from
    seed-0 parameters to oracle targets made with seed-42 parameters."""
    if not with_oracle:
        return None
    import oracle
    from paper_2604_20295_gb300 import fit as F
    sc = I.sphere_press_scene(1024, seed=7)
    tht = I.make_params(42)
    target = oracle.forward(sc, tht)["disp"]
    h = F.fit(sc, theta0, target, iters=200, lr=1e-3)
    err = {k: float(np.linalg.norm(h["params"][a:a + n] - tht[a:a + n]) /
                    max(np.linalg.norm(tht[a:a + n]), 1e-30))
           for k, (a, n, _) in I.param_slices().items()}
    err0 = {k: float(np.linalg.norm(theta0[a:a + n] - tht[a:a + n]) /
                     max(np.linalg.norm(tht[a:a + n]), 1e-30))
            for k, (a, n, _) in I.param_slices().items()}
    return {"workload": "1024 envs x sphere-press 16x16, Adam lr 1e-3, 200 iterations",
            "loss_first": h["loss"][0], "loss_last": h["loss"][-1],
            "norm_first": h["norm"][0], "norm_last": h["norm"][-1],
            "alpha_start": float(theta0[0]), "alpha_end": h["alpha"][-1],
            "alpha_target": float(tht[0]), "param_rel_error": err,
            "param_rel_error_start": err0, "seconds": h["seconds"]}


def config_fit_at_scale(I, theta0, with_oracle):
    """Eq. 5 calibration on the hand layout at its full size (4,096 envs, 18.9 M nodes):
    Adam over 200 iterations from seed-0 parameters to oracle targets made with seed-42
    parameters, with the passive-node RMS error on held-out envs (another seed) before and
    after the fit next to the parameter errors."""
    if not with_oracle:
        return None
    import oracle
    from paper_2604_20295_gb300 import fit as F
    sc = I.hand_scene(4096, seed=2)
    held = I.hand_scene(256, seed=99)
    tht = I.make_params(42)
    t0 = time.perf_counter()
    target = oracle.forward(sc, tht)["disp"]
    target_h = oracle.forward(held, tht)["disp"]
    t_oracle = time.perf_counter() - t0
    h = F.fit(sc, theta0, target, iters=200, lr=1e-3)
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return {"workload": "hand layout 4096 envs (18.9 M nodes), Adam lr 1e-3, 200 iterations; "
                        "held-out: 256 envs of another seed",
            "loss_first": h["loss"][0], "loss_last": h["loss"][-1],
            "alpha_start": float(theta0[0]), "alpha_end": h["alpha"][-1],
            "alpha_target": float(tht[0]),
            "alpha_rel_error_start": abs(float(theta0[0]) - float(tht[0])) / float(tht[0]),
            "alpha_rel_error_end": abs(h["alpha"][-1] - float(tht[0])) / float(tht[0]),
            "param_rel_error_start": rel(theta0, tht), "param_rel_error_end": rel(h["params"], tht),
            "heldout_passive_rms_mm_start": F.passive_rms(held, theta0, target_h),
            "heldout_passive_rms_mm_end": F.passive_rms(held, h["params"], target_h),
            "fit_seconds": h["seconds"], "ms_per_iteration": 1e3 * h["seconds"] / 201,
            "oracle_target_seconds": t_oracle}


def config_mesh(X, I, torch, dev, stream, flush, theta, with_oracle):
    """Mesh contact in the step: the hand layout (4,096 envs, 18.9 M nodes) pressed into four
    seeded rock meshes (1,280 triangles each), through the C ABI: the BF16 step and the FP32
    batched step with their kernels, and (with the oracle) the error of the BF16 step on a
    sample of envs against the FP64 oracle's mesh contact."""
    sc = I.mesh_scene(4096, seed=2)
    kw = dict(want_mask=True, want_pen=False, want_count=True)
    out = {"workload": "hand layout 4096 envs x rock meshes (4 x 1280 triangles)",
           "nodes_per_step": sc.total_nodes}
    for name, prec in (("bf16_batched", X.PREC_BF16), ("fp32_batched", X.PREC_FP32)):
        sim = X.TactileSim(sc, device=dev)
        try:
            sim.set_model(theta, X.MODE_FULL, prec, X.ALGO_BATCHED)
            sim.set_meshes()
            for _ in range(3):
                sim.step(**kw)
            torch.cuda.synchronize()
            X.etac_enable_timing(sim.ctx, True)
            ms = timed_steps(sim, 5, stream, flush, torch, kw)
            kt = X.etac_kernel_times(sim.ctx)
            X.etac_enable_timing(sim.ctx, False)
            out[name] = {"ms_per_step": sum(ms) / len(ms),
                         "node_steps_per_s": sc.total_nodes * 1e3 / (sum(ms) / len(ms)),
                         "kernels_ms": {k: v[1] / max(v[0], 1) for k, v in kt.items()},
                         "active_fraction": float(sim.mask.float().mean())}
            if with_oracle and prec == X.PREC_BF16:
                import oracle
                envs = np.sort(np.random.default_rng(3).choice(sc.num_envs, 32, replace=False))
                sub = sc.subset(envs)
                offs = sc.node_offsets
                idx = np.concatenate([np.arange(offs[e * 6], offs[e * 6 + 6]) for e in envs])
                ref = oracle.forward(sub, theta, mask_override=sim.mask.cpu().numpy()[idx])
                got = sim.disp.cpu().numpy()[idx].astype(np.float64)
                d = np.linalg.norm(got - ref["disp"], axis=1)
                out[name]["error_vs_oracle"] = dict(
                    max_abs_mm=float(d.max()), rms_mm=float(np.sqrt((d ** 2).mean())),
                    envs=len(envs),
                    mask_mismatch_nodes=int((oracle.forward(sub, theta)["mask"] !=
                                             sim.mask.cpu().numpy()[idx]).sum()))
        finally:
            sim.close()
    return out


def config_regressor(X, I, torch, dev, stream, theta, with_oracle):
    """The real-to-sim taxel regressor (appendix "Modeling Real Sensors") on the BF16 step's
    displacement field of the hand layout, 4,096 envs (18.9 M nodes, 24,576 pads), through the
    C ABI: the tensor-core path (per-node layers in BF16 with FP32 accumulation) per call and
    per kernel, its rate against the measured BF16 tensor peak (279,936 FLOP per node in the
    per-node layers), and (with the oracle) its error on three envs against the FP64 oracle,
    on the FP32 weights and on the same weights rounded to BF16.  The field (226 MB) is larger
    than L2, so calls are timed back to back."""
    sc = I.hand_scene(4096, seed=2)
    rp = I.make_regressor_params(0)
    sim = X.TactileSim(sc, device=dev)
    out = {"workload": "hand layout 4096 envs (18.9 M nodes, 24,576 pads), seeded regressor "
                       "weights, BF16 step field"}
    try:
        sim.set_model(theta, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        disp = sim.step().clone()
        rpt = torch.as_tensor(rp, device=dev)
        for _ in range(3):
            sim.regress(rpt, disp=disp, want_attn=False)
        torch.cuda.synchronize()
        X.etac_enable_timing(sim.ctx, True)
        reps = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sim.regress(rpt, disp=disp, want_attn=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        kt = X.etac_kernel_times(sim.ctx)
        X.etac_enable_timing(sim.ctx, False)
        assert sim.poll_status() == 0, "regressor status"
        y, a = sim.regress(rpt, disp=disp)
        torch.cuda.synchronize()
        envs = [0, 2047, 4095]
        P, offs = sc.pads_per_env, sc.node_offsets
        rows = np.concatenate([np.arange(offs[e * P], offs[(e + 1) * P]) for e in envs])
        pads = np.concatenate([np.arange(e * P, (e + 1) * P) for e in envs])
        d_s = disp.cpu().numpy()[rows].astype(np.float64)
        y_s = y.cpu().numpy()[pads].astype(np.float64)
    finally:
        sim.close()
    flops = 279936.0 * sc.total_nodes
    peaks, src = _peaks()
    k_ms = kt["regress_tc_kernel"][1] / max(kt["regress_tc_kernel"][0], 1)
    ach = flops / k_ms / 1e9
    out.update({"ms_per_call": ms, "node_per_s": sc.total_nodes * 1e3 / ms,
                "kernels_ms": {k: v[1] / max(v[0], 1) for k, v in kt.items()},
                "roofline": {"bound": "tensor", "kernel": "regress_tc_kernel",
                             "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                             "frac": ach / peaks["bf16_tflops"],
                             "peak_source": f"{src} bf16_tflops (burst)",
                             "flop_per_node": 279936}})
    if with_oracle:
        import oracle
        sub = sc.subset(envs)
        rp64 = rp.astype(np.float64)
        rpb = rp64.copy()
        sl = I.regressor_param_slices()
        for k in ("WR1", "WR2", "WR3", "WR4", "WA1"):
            s0, n, _ = sl[k]
            rpb[s0:s0 + n] = torch.as_tensor(rp[s0:s0 + n]).to(torch.bfloat16).double().numpy()
        err = {}
        for name, w in (("fp32_weights", rp64), ("bf16_weights", rpb)):
            ref = oracle.regress(sub, d_s, w)["taxels"]
            scale = np.abs(ref).max(axis=1)
            err[name] = {"max_abs": float(np.abs(y_s - ref).max()),
                         "max_pad_rel": float((np.abs(y_s - ref).max(axis=1) / scale).max())}
        out["error_vs_oracle"] = dict(err, envs=len(envs), pads=len(pads))
    return out


def config_c4_fd(X, I, torch, dev):
    """The reverse mode against FP64 central differences (h = 1e-6) of the GPU FP64 forward:
    1 env, one 8x8 flat pad, each primitive; the 6 pose components, alpha and 24 sampled
    weights.  The adjoint is the batched FP32 reverse mode (the one timed above)."""
    h = 1e-6
    out = {"workload": "1 env x 8x8 flat pad per primitive, FP64 central differences, h = 1e-6"}
    worst = 0.0
    for name, ot in (("sphere", I.OBJ_SPHERE), ("box", I.OBJ_BOX), ("cylinder", I.OBJ_CYLINDER),
                     ("capsule", I.OBJ_CAPSULE)):
        sc = I.grad_scene(ot, seed=0)
        th = I.make_params(7).astype(np.float64)
        G = np.random.default_rng(5).normal(size=(sc.total_nodes, 3))
        sim = X.TactileSim(sc, device=dev)
        try:
            sim.set_model(th.astype(np.float32), X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
            sim.step()
            g = sim.backward(torch.as_tensor(np.asarray(G, np.float32), device=dev))
            torch.cuda.synchronize()
            adj_pose = g["obj_pose"].cpu().numpy().astype(np.float64)[0]
            adj_par = g["params"].cpu().numpy().astype(np.float64)

            def loss(pose, theta):
                disp = torch.zeros(sc.total_nodes, 3, dtype=torch.float64, device=dev)
                ten = [torch.as_tensor(np.asarray(v, np.float64), device=dev)
                       for v in (sc.obj_dims, pose, sc.pad_pose, theta)]
                X.etac_forward_f64(sim.ctx, X.etac_model_desc(64, 0, 0, 0), sim.obj_type.data_ptr(),
                                   *[t.data_ptr() for t in ten], disp.data_ptr(),
                                   torch.cuda.current_stream(dev).cuda_stream)
                torch.cuda.synchronize()
                return float((disp.cpu().numpy() * G).sum())

            op = sc.obj_pose.astype(np.float64)
            fd_pose = np.zeros(6)
            for a in range(6):
                def pose(sgn):
                    o = op.copy()
                    if a < 3:
                        o[a] += sgn * h
                    else:
                        ax = np.zeros(3)
                        ax[a - 3] = 1.0
                        o[3:] = I._qmul(I._axis_angle(ax, sgn * h), o[3:] / np.linalg.norm(o[3:]))
                    return o
                fd_pose[a] = (loss(pose(1), th) - loss(pose(-1), th)) / (2 * h)
            idx = [0] + list(np.random.default_rng(11).choice(np.arange(1, th.size), 24, replace=False))
            fd_par = np.array([(loss(op, th + h * (np.arange(th.size) == k)) -
                                loss(op, th - h * (np.arange(th.size) == k))) / (2 * h) for k in idx])
        finally:
            sim.close()
        ep = float(np.abs(adj_pose - fd_pose).max() / max(np.abs(fd_pose).max(), 1e-3))
        eq = float(np.abs(adj_par[idx] - fd_par).max() / max(np.abs(fd_par).max(), 1e-3))
        out[name] = {"pose_max_rel_err": ep, "params_max_rel_err": eq}
        worst = max(worst, ep, eq)
    out["worst_max_rel_err"] = worst
    return out


def config_c5_continuous(X, I, torch, dev, stream, flush, theta, peaks, with_oracle):
    """The continuous-pitch variant of the uneven workload: 2,048 envs x 6 flat pads of
    8x8 .. 64x64 nodes, each pad with its own pitch ~U[0.5, 2] mm (12,288 pad types, so no
    Omega table is shared: at 16,384 envs the tables would need 1.7 TB), 1-3 primitives per
    env.  The batched FP32 step with Omega on the fly (the library's own choice here), timed
    per step and per kernel, its rate over the propagation pairs against the special-function
    pipe (each pair takes one sqrt and one exp), and its error on sampled envs against the
    oracle.  2,048 of the 16,384 envs keep the per-type node tables at 24 GB."""
    sc = I.uneven_continuous_scene(2048, seed=5)
    sim = X.TactileSim(sc, device=dev)
    out = {"workload": "uneven-continuous-pitch-2048env-6pads-8x8..64x64 (12,288 pad types)",
           "nodes_per_step": sc.total_nodes}
    try:
        sim.set_model(theta, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        kw = dict(want_mask=False, want_pen=False, want_count=True)
        for _ in range(3):
            sim.step(**kw)
        torch.cuda.synchronize()
        counts = sim.count.cpu().numpy()
        work = algorithmic_work(sc, counts)
        X.etac_enable_timing(sim.ctx, True)
        ms = timed_steps(sim, 5, stream, flush, torch, kw)
        kt = X.etac_kernel_times(sim.ctx)
        X.etac_enable_timing(sim.ctx, False)
        fwd_ms = sum(ms) / len(ms)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = peaks.get("sm_max_mhz", 2070.0)
        sfu_peak = nsm * 16 * mhz * 1e6 / 1e12   # special-function ops per second (x 1e12)
        k_ms = kt["batched_forward_kernel<fp32>"][1] / max(kt["batched_forward_kernel<fp32>"][0], 1)
        ach = 2.0 * work["pairs"] / k_ms / 1e9
        out.update({"omega": "on the fly (the tables would exceed the 4 GiB cache limit)",
                    "fwd_ms": fwd_ms, "fwd_node_steps_per_s": sc.total_nodes * 1e3 / fwd_ms,
                    "active_fraction": work["active"] / sc.total_nodes,
                    "pairs": work["pairs"],
                    "kernels_ms": {k: v[1] / max(v[0], 1) for k, v in kt.items()},
                    "roofline": {"bound": "alu", "kernel": "batched_forward_kernel<fp32>",
                                 "achieved": ach, "peak": sfu_peak, "unit": "Tops/s",
                                 "frac": ach / sfu_peak,
                                 "peak_source": f"derived: {nsm} SMs x 16 special-function "
                                                f"ops/clk x {mhz} MHz; 2 ops (sqrt, exp) per "
                                                f"(passive, active) pair"}})
        if with_oracle:
            import oracle
            envs = np.sort(np.random.default_rng(9).choice(sc.num_envs, 16, replace=False))
            sub = sc.subset(envs)
            sim.step(want_mask=True, want_pen=False, want_count=True)
            torch.cuda.synchronize()
            offs = sc.node_offsets
            idx = np.concatenate([np.arange(offs[e * 6], offs[e * 6 + 6]) for e in envs])
            ref = oracle.forward(sub, theta)
            out["error_vs_oracle"] = dict(_stats(sim.disp.cpu().numpy()[idx], ref["disp"],
                                                 sim.mask.cpu().numpy()[idx], ref["mask"]),
                                          envs=len(envs))
    finally:
        sim.close()
    return out


def config_c5(X, I, torch, dev, stream, flush, theta, peaks, with_oracle):
    """Scale and unevenness: 16,384 envs x 6 flat pads of 8x8 .. 64x64 nodes (16 pad types),
    1-3 primitives per env; BF16 forward and FP32 reverse mode."""
    sc = I.uneven_scene(16384, seed=5)
    sim = X.TactileSim(sc, device=dev)
    sim.set_model(theta, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
    kw = dict(want_mask=False, want_pen=False, want_count=True)
    for _ in range(3):
        sim.step(**kw)
    torch.cuda.synchronize()
    counts = sim.count.cpu().numpy()
    work = algorithmic_work(sc, counts)
    X.etac_enable_timing(sim.ctx, True)
    ms = timed_steps(sim, 5, stream, flush, torch, kw)
    kt = X.etac_kernel_times(sim.ctx)
    fwd_ms = sum(ms) / len(ms)
    G = torch.randn(sim.disp.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(4))
    sim.step(**kw)
    for _ in range(2):
        sim.backward(G)
    torch.cuda.synchronize()
    bms = []
    for _ in range(3):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.backward(G)
        e1.record(stream)
        torch.cuda.synchronize()
        bms.append(e0.elapsed_time(e1))
    kt2 = X.etac_kernel_times(sim.ctx)
    X.etac_enable_timing(sim.ctx, False)
    nodes = sc.total_nodes
    gk = kt.get("prop_gemm_kernel", (1, 0.0))
    t_gemm = gk[1] / max(gk[0], 1) / 1e3
    alg = 6.0 * work["pairs"] + 2.0 * 3 * H * work["passive"]
    exe = executed_gemm_flops(sc)
    out = {"workload": "uneven-16384env-6pads-8x8..64x64-16types", "nodes_per_step": nodes,
           "fwd_ms": fwd_ms, "fwd_node_steps_per_s": nodes * 1e3 / fwd_ms,
           "bwd_ms": sum(bms) / len(bms), "bwd_fwd": sum(bms) / len(bms) / fwd_ms,
           "active_fraction": work["active"] / nodes,
           "fwd_kernels": {k: v[1] / max(v[0], 1) for k, v in kt.items()},
           "bwd_kernels": {k: v[1] / max(v[0], 1) for k, v in kt2.items()},
           "roofline_prop_gemm": {"bound": "tensor", "achieved": alg / t_gemm / 1e12,
                                  "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                                  "frac": alg / t_gemm / 1e12 / peaks["bf16_tflops"],
                                  "executed_dense_tflops": exe / t_gemm / 1e12,
                                  "executed_frac": exe / t_gemm / 1e12 / peaks["bf16_tflops"]},
           "roofline_step_hbm": {"bound": "hbm", "achieved": work["bytes_out"] * 1e3 / fwd_ms / 1e9,
                                 "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": work["bytes_out"] * 1e3 / fwd_ms / 1e9 / peaks["hbm_gbs"],
                                 "note": "12 B of displacement out per node over the whole step"}}
    if with_oracle:
        import oracle
        envs = np.sort(np.random.default_rng(9).choice(sc.num_envs, 48, replace=False))
        sub = sc.subset(envs)
        sim.step(want_mask=True, want_pen=False, want_count=True)
        torch.cuda.synchronize()
        offs = sc.node_offsets
        idx = np.concatenate([np.arange(offs[e * 6], offs[e * 6 + 6]) for e in envs])
        t0 = time.perf_counter()
        ref = oracle.forward(sub, theta)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": sub.total_nodes / dt, "unit": UNIT, "cores": cpu_cores(),
                               "kind": "oracle",
                               "sample": f"{len(envs)} random envs ({sub.total_nodes} nodes) of "
                                         f"this workload, FP64 forward, OpenMP over pads, "
                                         f"{dt:.1f} s"}
        out["error_vs_oracle"] = dict(_stats(sim.disp.cpu().numpy()[idx], ref["disp"],
                                             sim.mask.cpu().numpy()[idx], ref["mask"]),
                                      envs=len(envs))
    sim.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="batched", choices=["plain", "batched"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--ref-envs", type=int, default=96)
    ap.add_argument("--cpu-envs", type=int, default=2048)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-bwd", action="store_true")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="streams the end-to-end read-back is split over")
    ap.add_argument("--no-graph", action="store_true",
                    help="time eager launches only (default: the step replayed from a CUDA graph)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile / block shapes instead of measuring them")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-pad BF16, calibration and 16,384-env uneven sections")
    ap.add_argument("--configs", default="all",
                    help="comma-separated names of the sections to run (c3, c4_fit, c4_fd, "
                         "fit_at_scale, mesh, regressor, c5, c5_continuous), or all")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    theta = I.make_params(0)
    scene = I.hand_scene(args.envs, seed=args.seed + 1000 * rank)

    if args.impl == "reference":
        return run_reference(args, scene, theta, rank, world)

    import torch
    from paper_2604_20295_gb300 import build as B
    from paper_2604_20295_gb300 import etac as X

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    algo = X.ALGO_BATCHED if args.algo == "batched" else X.ALGO_PLAIN
    prec = X.PREC_BF16 if args.precision == "bf16" else X.PREC_FP32
    sim = X.TactileSim(scene, device=dev)
    sim.set_model(theta, X.MODE_FULL, prec, algo)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    step_kw = dict(want_mask=False, want_pen=False, want_count=True)

    tuning = None
    if not args.no_autotune and algo == X.ALGO_BATCHED:
        gt = torch.randn(sim.disp.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
        tuning = sim.autotune(None if args.no_bwd else gt)
        del gt

    clocks = Clocks(local)
    clocks.start()    # sampled from before warm-up until after the timed region
    for _ in range(args.warmup):
        sim.step(**step_kw)
    torch.cuda.synchronize()
    counts = sim.count.cpu().numpy()
    work = algorithmic_work(scene, counts)

    # ---- device-timed region: K steps, per-kernel events on the launching stream
    X.etac_enable_timing(sim.ctx, True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    step_ms = timed_steps(sim, args.steps, stream, flush, torch, step_kw)
    if pg:
        pg.barrier()
    ktimes = X.etac_kernel_times(sim.ctx)
    X.etac_enable_timing(sim.ctx, False)

    nodes = scene.total_nodes
    eager_s = max_over_ranks(sum(step_ms) / 1e3, pg, dev)
    eager = {"value": job_rate(nodes, args.steps, world, eager_s), "unit": UNIT,
             "ms_per_step": 1e3 * eager_s / args.steps}

    # ---- the same step captured once in a CUDA graph and replayed K times (the headline)
    graph = None
    if not args.no_graph:
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            sim.step(**step_kw)
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg, stream=gs):
                sim.step(**step_kw)
        stream.wait_stream(gs)
        for _ in range(max(3, args.warmup)):
            cg.replay()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            cg.replay()
            ends[k].record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        g_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        graph_s = max_over_ranks(sum(g_ms) / 1e3, pg, dev)
        graph = {"value": job_rate(nodes, args.steps, world, graph_s), "unit": UNIT,
                 "ms_per_step": 1e3 * graph_s / args.steps, "launches_per_step":
                 int(sum(v[0] for v in ktimes.values()) // max(args.steps, 1))}
        step_ms = g_ms
        # untimed replays of the same step for about a second, so that the clock sampler
        # (one nvidia-smi reading per 200 ms) sees the GPU under this load several times: the
        # timed steps alone last a few milliseconds
        soak = max(1, int(1.0 / max(g_ms[0] / 1e3, 1e-5)))
        for _ in range(soak):
            cg.replay()
        torch.cuda.synchronize()
        del cg
    clk = clocks.stop()
    if clk is not None:
        clk["sampled_over"] = ("warm-up, the timed steps and about 1 s of untimed replays of the "
                               "same step right after them")
    head = graph or eager
    value = head["value"]
    ms_per_step = head["ms_per_step"]

    # ---- end to end through the public API with host buffers: every step copies its inputs
    # from pinned host memory and its whole displacement back to pinned host memory.  Two
    # output buffers alternate, so the read-back of step k (on a copy stream) overlaps step
    # k + 1; a buffer is rewritten only after its copy has finished.
    e2e = None
    if not args.no_e2e:
        # the pinned buffers are allocated (and so placed) from the CPUs of the GPU's own NUMA
        # node when the system names them; the process's CPU set is restored afterwards
        local = gpu_local_cpus(torch, dev)
        saved = os.sched_getaffinity(0) if local else None
        try:
            if local:
                os.sched_setaffinity(0, local)
            pin = lambda a: torch.as_tensor(a).pin_memory()
            h_in = [pin(scene.obj_type), pin(scene.obj_dims), pin(scene.obj_pose),
                    pin(scene.pad_pose)]
            h_out = [torch.empty(sim.disp.shape, dtype=torch.float32, pin_memory=True)
                     for _ in range(2)]
        finally:
            if saved:
                os.sched_setaffinity(0, saved)
        d_in = [sim.obj_type, sim.obj_dims, sim.obj_pose, sim.pad_pose]
        d_out = [sim.disp, torch.empty_like(sim.disp)]
        h2d = sum(t.numel() * t.element_size() for t in h_in)
        d2h = h_out[0].numel() * 4
        ke = max(20, args.steps)   # enough steps that filling the copy pipeline is amortised
        ncs = max(1, args.copy_streams)
        css = [torch.cuda.Stream(dev) for _ in range(ncs)]
        rows = sim.disp.shape[0]
        cuts = [rows * c // (2 * ncs) for c in range(2 * ncs + 1)]   # 2 chunks per copy stream
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [[torch.cuda.Event() for _ in range(ncs)] for _ in range(2)]
        # the link alone: the same read-back with no step beside it (3 copies, events on the
        # copy stream), so that the end-to-end rate can be put against what the link carries
        torch.cuda.synchronize()
        link = []
        for b in range(2):
            l0 = torch.cuda.Event(enable_timing=True)
            l1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(css[0]):
                h_out[b].copy_(d_out[b], non_blocking=True)
                l0.record(css[0])
                for _ in range(3):
                    h_out[b].copy_(d_out[b], non_blocking=True)
                l1.record(css[0])
            torch.cuda.synchronize()
            link.append(3 * d2h / (l0.elapsed_time(l1) * 1e6))
        link_gbs = min(link)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(ke):
            b = k & 1
            for d, h in zip(d_in, h_in):
                d.copy_(h, non_blocking=True)
            if k >= 2:
                for ev in done[b]:
                    stream.wait_event(ev)
            sim.step(disp=d_out[b], **step_kw)
            ready[b].record(stream)
            for j, cs in enumerate(css):
                cs.wait_event(ready[b])
                with torch.cuda.stream(cs):
                    for c in (2 * j, 2 * j + 1):
                        h_out[b][cuts[c]:cuts[c + 1]].copy_(d_out[b][cuts[c]:cuts[c + 1]],
                                                            non_blocking=True)
                done[b][j].record(cs)
        for cs in css:
            stream.wait_stream(cs)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, pg, dev)
        same = bool(torch.equal(h_out[(ke - 1) & 1], d_out[(ke - 1) & 1].cpu()))
        e2e = {"value": job_rate(nodes, ke, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ke, "ms_per_step": 1e3 * e2e_s / ke,
               "pipelining": f"read-back of step k overlaps step k + 1 (two output buffers, "
                             f"{ncs} copy stream(s), {2 * ncs} chunks)",
               "readback_matches_device": same,
               "d2h_link_gbs": link_gbs,
               "d2h_link_gbs_per_buffer": link,
               "host_buffers_cpus": (f"{len(local)} CPUs local to the GPU" if local
                                     else "the process's CPU set"),
               "d2h_frac_of_link": d2h * ke / e2e_s / 1e9 / link_gbs}

    # ---- the other rungs on the same GPU and scene (the metric compares BF16 batched with
    # FP32 plain; FP32 batched is the intermediate rung)
    compare = {}
    if not args.no_compare:
        for name, a2, p2, k2 in (("fp32_plain", X.ALGO_PLAIN, X.PREC_FP32, 3),
                                 ("fp32_batched", X.ALGO_BATCHED, X.PREC_FP32, 5),
                                 ("bf16_batched", X.ALGO_BATCHED, X.PREC_BF16, 5)):
            if (a2, p2) == (algo, prec):
                continue
            s2 = X.TactileSim(scene, device=dev)
            s2.set_model(theta, X.MODE_FULL, p2, a2)
            for _ in range(2):
                s2.step(**step_kw)
            ms = timed_steps(s2, k2, stream, flush, torch, step_kw)
            compare[name] = {"value": nodes * 1e3 / (sum(ms) / k2), "unit": UNIT,
                             "ms_per_step": sum(ms) / k2, "steps": k2}
            s2.close()
        compare[f"{args.precision}_{args.algo}"] = {"value": value, "unit": UNIT,
                                                    "ms_per_step": ms_per_step}

    peaks_early, _ = _peaks()
    nsm_early = torch.cuda.get_device_properties(dev).multi_processor_count
    # ---- reverse mode (FP32 adjoint): bwd/fwd on this workload and on the 1,024-env layout
    # of 16x16 flat pads (forward FP32 batched there)
    bwd = None
    if not args.no_bwd:
        def time_bwd(s_, G_, k):
            for _ in range(2):
                s_.backward(G_)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(k):
                flush.fill_(1)
                e0.record(stream)
                s_.backward(G_)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return sum(ms) / k
        gen = torch.Generator(device=dev).manual_seed(3)
        G = torch.randn(sim.disp.shape, device=dev, generator=gen)
        sim.step(**step_kw)
        b_ms = time_bwd(sim, G, 3)
        # per-stage times of one more reverse pass (events around each stage's launches)
        X.etac_enable_timing(sim.ctx, True)
        flush.fill_(2)
        sim.backward(G)
        torch.cuda.synchronize()
        bk = X.etac_kernel_times(sim.ctx)
        X.etac_enable_timing(sim.ctx, False)
        bwd_stages = bwd_rooflines(bk, scene, work, peaks_early, nsm_early)
        small = I.sphere_press_scene(1024, seed=7)
        s4 = X.TactileSim(small, device=dev)
        s4.set_model(theta, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        for _ in range(3):
            s4.step(**step_kw)
        f4 = timed_steps(s4, 10, stream, flush, torch, step_kw)
        G4 = torch.randn(s4.disp.shape, device=dev, generator=gen)
        b4 = time_bwd(s4, G4, 10)
        s4.close()
        bwd = {"workload": {"fwd_ms": ms_per_step, "bwd_ms": b_ms, "bwd_fwd": b_ms / ms_per_step,
                            "fwd": f"{args.precision} {args.algo}", "bwd": "fp32 adjoint",
                            "stages": bwd_stages},
               "flat16x16_1024env": {"fwd_ms": sum(f4) / len(f4), "bwd_ms": b4,
                                     "bwd_fwd": b4 / (sum(f4) / len(f4)),
                                     "fwd": "fp32 batched", "bwd": "fp32 adjoint"}}

    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    kern = {k: {"launches": v[0], "ms_per_launch": v[1] / max(v[0], 1)} for k, v in ktimes.items()}
    roof_all = None
    if args.algo == "plain":
        name = "plain_forward_kernel<float>"
        fma_peak = nsm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        t_launch = kern[name]["ms_per_launch"] / 1e3
        achieved = work["literal_flops"] / t_launch / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fma_peak, "unit": "TFLOP/s",
                "frac": achieved / fma_peak, "traffic": None, "kernel": name,
                "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x 2 x "
                               f"{peaks.get('sm_max_mhz', 2070.0)} MHz"}
    elif args.precision == "fp32":
        name = "batched_forward_kernel<fp32>"
        t_launch = kern[name]["ms_per_launch"] / 1e3
        achieved = work["bytes_out"] / t_launch / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": name,
                "peak_source": f"{peak_src} (MEASURED_PEAKS hbm_gbs)"}
    else:
        # per-kernel rooflines of the BF16 step; the top-level entry is the kernel with the
        # largest share of the step
        full_size = scene.num_envs == 4096 and args.seed == 2   # the workload the counters are of
        peak = peaks["bf16_tflops"]
        per = {}
        t = kern["front_contact_kernel"]["ms_per_launch"] / 1e3
        # the method's contraction on this kernel: the encoder of the active nodes, factored
        # (E1 on the 3 u_hat inputs, the geometric part being a per-type table, then E2):
        # 2 (3 x 64 + 64 x 64) = 8,576 FLOP per active node; the FP32 SDF and max-pool work is
        # not tensor work and is left out of this numerator
        alg = 2.0 * (3 * H + H * H) * work["active"]
        per["front_contact_kernel"] = {
            "bound": "tensor", "achieved": alg / t / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": alg / t / 1e12 / peak, "traffic": full_size and traffic_for("front_contact_kernel") or None,
            "ms": t * 1e3, "peak_source": f"{peak_src} bf16_tflops (burst)",
            "note": "factored encoder FLOPs of the active nodes (8,576 per node) over the "
                    "kernel time; the kernel is latency- and issue-bound (see issue), and its "
                    "HBM bytes are small (12 B per active node + 4 B per pad)"}
        ipn = instr_per_node("front_contact_kernel")
        if ipn is not None:
            # the bound that explains this kernel: instruction issue (one warp instruction per
            # scheduler per cycle: SMs x 4 x max SM clock); its tensor figure stays beside it
            issue_peak = nsm * 4 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9
            ach = ipn * nodes / t / 1e9
            tensor = per["front_contact_kernel"]
            per["front_contact_kernel"] = {
                "bound": "issue", "achieved": ach, "peak": issue_peak,
                "unit": "G warp-instructions/s", "frac": ach / issue_peak,
                "traffic": tensor["traffic"], "ms": tensor["ms"],
                "warp_instructions_per_node": ipn,
                "peak_source": f"derived: {nsm} SMs x 4 schedulers x "
                               f"{peaks.get('sm_max_mhz', 2070.0)} MHz",
                "note": "instruction issue binds this kernel (contact classification, the "
                        "mma.sync encoder drains and the max-pool walk); achieved = ncu warp "
                        "instructions per node x nodes / event time; the rest of its cycles "
                        "are latency (instruction fetch and mma.sync dependency stalls)",
                "tensor": {k: tensor[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                  "peak_source", "note")}}
        t = kern["prop_gemm_kernel"]["ms_per_launch"] / 1e3
        alg = 6.0 * work["pairs"] + 2.0 * 3 * H * work["passive"]
        exe = executed_gemm_flops(scene)
        per["prop_gemm_kernel"] = {
            "bound": "tensor", "achieved": alg / t / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": alg / t / 1e12 / peak, "traffic": full_size and traffic_for("prop_gemm_kernel") or None,
            "ms": t * 1e3, "executed_dense_tflops": exe / t / 1e12,
            "executed_frac": exe / t / 1e12 / peak,
            "peak_source": f"{peak_src} bf16_tflops (burst)",
            "note": "achieved counts the Eq. 1 contraction over (passive, active) pairs and "
                    "the decoder output layer; the kernel executes the dense per-type "
                    "contraction (executed_dense_tflops)"}
        t = kern["front_global_kernel"]["ms_per_launch"] / 1e3
        npads = scene.num_envs * scene.pads_per_env
        byts = npads * (4 * H + 2 * H + 16)               # g0 in, -beta (BF16) and (c0, m) out
        per["front_global_kernel"] = {
            "bound": "hbm", "achieved": byts / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": byts / t / 1e9 / peaks["hbm_gbs"],
            "traffic": full_size and traffic_for("front_global_kernel") or None, "ms": t * 1e3,
            "peak_source": f"{peak_src} hbm_gbs"}
        name = max(per, key=lambda k: per[k]["ms"])
        roof = dict(per[name], kernel=name)
        roof_all = per
    cpu = None
    err = None
    if not args.no_cpu and rank == 0:
        envs = np.sort(np.random.default_rng(7).choice(scene.num_envs,
                                                       min(args.cpu_envs, scene.num_envs),
                                                       replace=False))
        import oracle
        sub = scene.subset(envs)
        t0 = time.perf_counter()
        ref = oracle.forward(sub, theta)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.total_nodes / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{len(envs)} random envs ({sub.total_nodes} nodes) of the workload, one "
                         f"forward step, FP64 C oracle, OpenMP over pads, {dt:.1f} s"}
        r1, dt1, nn1 = oracle_single_core(scene, theta, envs[:16])
        cpu["single_core"] = {"value": r1, "unit": UNIT, "cores": 1,
                              "sample": f"{min(len(envs), 16)} of those envs ({nn1} nodes), one "
                                        f"thread, {dt1:.1f} s"}
        # stated error of this run's output on the same envs (mask-matched pads)
        sim.step(want_mask=True, want_pen=False, want_count=True)
        torch.cuda.synchronize()
        offs = scene.node_offsets
        idx = np.concatenate([np.arange(offs[e * 6], offs[e * 6 + 6]) for e in envs])
        got = sim.disp.cpu().numpy()[idx].astype(np.float64)
        gm = sim.mask.cpu().numpy()[idx]
        same = gm == ref["mask"]
        d = np.linalg.norm(got - ref["disp"], axis=1)
        so = sub.node_offsets
        pad_err = np.maximum.reduceat(d, so[:-1])
        pad_scale = np.maximum.reduceat(np.linalg.norm(ref["disp"], axis=1), so[:-1])
        err = {"max_abs_mm": float(d.max()), "rms_mm": float(np.sqrt((d ** 2).mean())),
               "max_pad_rel": float((pad_err / np.maximum(pad_scale, 1e-30)).max()),
               "mask_mismatch_nodes": int((~same).sum()), "envs": len(envs)}

    configs = None
    if not args.no_configs and rank == 0:
        sim.close()
        sim = None
        with_oracle = not args.no_cpu
        sections = {
            "c3": ("c3_bf16_single_pad",
                   lambda: config_c3(X, I, torch, dev, stream, flush, theta, with_oracle)),
            "c4_fit": ("c4_fit", lambda: config_c4_fit(I, theta, with_oracle)),
            "c4_fd": ("c4_fd_check", lambda: config_c4_fd(X, I, torch, dev)),
            "fit_at_scale": ("fit_at_scale_hand4096",
                             lambda: config_fit_at_scale(I, theta, with_oracle)),
            "mesh": ("mesh_hand4096",
                     lambda: config_mesh(X, I, torch, dev, stream, flush, theta, with_oracle)),
            "regressor": ("regressor_hand4096",
                          lambda: config_regressor(X, I, torch, dev, stream, theta, with_oracle)),
            "c5": ("c5_uneven_16384",
                   lambda: config_c5(X, I, torch, dev, stream, flush, theta, peaks, with_oracle)),
            "c5_continuous": ("c5_continuous_pitch_2048",
                              lambda: config_c5_continuous(X, I, torch, dev, stream, flush, theta,
                                                           peaks, with_oracle))}
        wanted = list(sections) if args.configs == "all" else args.configs.split(",")
        configs = {sections[k][0]: sections[k][1]() for k in wanted}

    # the metric's two comparisons, early in the line: BF16 batched over FP32 plain on this
    # workload, and the reverse mode's time over the forward's
    ratio_plain = (value / compare["fp32_plain"]["value"]
                   if compare and "fp32_plain" in compare else None)
    bwd_fwd_main = bwd["workload"]["bwd_fwd"] if bwd and "workload" in bwd else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "bf16_vs_fp32_plain": ratio_plain, "bwd_fwd": bwd_fwd_main,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == X.PREC_BF16 else "f32",
            "data": "synthetic", "config": dict(workload_config(args, scene), tuning=tuning),
            "roofline": roof,
            "roofline_by_kernel": roof_all,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(sum(v["launches"] for v in kern.values())),
            "eager": eager, "graph": graph,
            "clocks": clk, "error_vs_oracle": err, "rungs": compare, "kernels": kern,
            "bwd_fwd_detail": bwd, "configs": configs,
            "active_fraction": work["active"] / nodes,
            "step_ms_min": min(step_ms), "step_ms_max": max(step_ms)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
