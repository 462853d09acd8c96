"""Benchmark: two-component D3Q19 lattice updates per second (GLUPS) of the full coupled time step on one
GB300, with the bulk stream + collide phase's fraction of the HBM roofline, an end-to-end figure through the C ABI
with host buffers, and the FP64 oracle timed on the host cores as a CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent replica of the workload
(the single-box problem does not shard); value = all ranks' lattice updates / max elapsed time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1904_11386_gb300 import inputs  # noqa: E402

# Algorithmic bytes per lattice update (both components): read and write 2 x 19 populations (4 bytes each in
# FP32 storage, 2 in FP16 or BF16), write rho^A and rho^B (FP32) and read them back (the Shan-Chen force needs
# the neighbours' densities of the same time level): 320 B, or 168 B with 16-bit populations.
BYTES_PER_LU = 2 * 19 * 4 * 2 + 2 * 4 + 2 * 4
BYTES_PER_LU_16 = 2 * 19 * 2 * 2 + 2 * 4 + 2 * 4
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2, "fp16dev": 3, "bf16dev": 4}
# error against the FP64 oracle of each 16-bit storage, as the tests bound it
STORAGE_ERROR = {
    "fp16": ("densities 1.3e-3, velocities 2.2e-3 of max|u|, vertices 2.5e-3 after 200 steps (32^3); mass offset "
             "4.7e-6, drift 2.0e-4 over 2000 steps (128^3, FP32 2.3e-4; measured with a colour offset four times "
             "the present one); tests/test_gpu_storage16.py"),
    "bf16": ("densities 2.0e-2, velocities 2.6e-2 of max|u|, vertices 2.0e-2 after 200 steps (32^3); mass offset "
             "1.5e-4, drift 1.5e-4 over 2000 steps (128^3, FP32 2.3e-4; measured with a colour offset four times "
             "the present one); tests/test_gpu_storage16.py"),
}


FALLBACK_HBM_GBS = 6800.0
# the headline metric, the same string on both arms (the oracle's line carries it too)
METRIC = ("2-component D3Q19 lattice updates per second, full coupled step (GLUPS); bulk stream+collide phase "
          "fraction of HBM roofline")


def bytes_per_lu(storage: str) -> int:
    return BYTES_PER_LU if storage == "fp32" else BYTES_PER_LU_16


def workload(name: str):
    if name == "adsorb128":
        return inputs.cfg_adsorb128(coupling=0), ("adsorb128: 128^3 D3Q19 x2 Shan-Chen, walls sheared 1e-4, "
                                                  "s=4 capsule R=12 (2562 vertices), half-way bounce-back, "
                                                  "colour 0.05, fresh nodes with mass correction")
    if name == "adsorb128-ibm":
        return inputs.cfg_adsorb128(coupling=1), ("adsorb128-ibm: same box and capsule with the 2-point "
                                                  "immersed-boundary coupling (colour 0)")
    if name == "parity32":
        return inputs.cfg_parity(coupling=1), "parity32-ibm2: 32^3, psi=rho, s=3 capsule R=6"
    if name == "batch48":
        return inputs.cfg_batch48(), ("batch48: 48 independent cubes with integer edges 40-72, each a flat "
                                      "interface with one s=3 capsule R=6 (642 vertices), colours over [-0.1, 0.1] "
                                      "x shear moduli {0.001, 0.003, 0.01, 0.03}, half-way bounce-back")
    if name == "droplet256":
        p = inputs.cfg_droplet256(n_caps=300, coupling=0)
        return p, (f"droplet256: 256^3 periodic two-component box, B droplet R=70 covered by {len(p.capsules)} s=3 "
                   "capsules R=8 (642 vertices each, softness beta=100) with colours +-0.05, half-way bounce-back, "
                   "repulsion")
    if name == "droplet128":
        p = inputs.cfg_droplet256(n_caps=40, coupling=0, n=128, R_drop=35.0)
        return p, (f"droplet128: 128^3 periodic two-component box, B droplet R=35 covered by {len(p.capsules)} s=3 "
                   "capsules R=8 with colours +-0.05, half-way bounce-back, repulsion")
    if name == "adjoint64":
        return inputs.cfg_adjoint64(coupling=1), ("adjoint64: 64^3 box between walls, flat interface, one s=3 "
                                                  "capsule R=8 (642 vertices) 4 above it, 2-point immersed "
                                                  "boundary; gradient of the capsule's centre-of-mass height "
                                                  "after 2000 steps w.r.t. kS, kB, kV, the initial vertices, G "
                                                  "and g, checkpoint every 100 steps")
    if name == "adjoint64-fluid":
        return inputs.cfg_adjoint(n=64, R_drop=16.0), ("adjoint64-fluid: 64^3 periodic two-component box, B "
                                                       "droplet R=16, gradient of the components' weighted "
                                                       "centres of mass after 2000 steps w.r.t. G, g and the "
                                                       "initial densities, checkpoint every 100 steps")
    if name == "fluid256":
        p = inputs.cfg_droplet256(n_caps=0, coupling=1)
        p.capsules = []
        return p, "fluid256: 256^3 periodic two-component droplet, no capsules"
    raise SystemExit(f"unknown workload {name}")


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                if isinstance(v, dict):
                    v = v.get("value", v.get("gbs"))
                return float(v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.file = None

    def start(self):
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def replica_max(x: float, ws: int, device: str = "cpu") -> float:
    """Max over all ranks of one rank's elapsed time (every rank calls it; ws = 1 returns x)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(nodes: int, steps: int, ws: int, seconds: float) -> float:
    """Whole-job lattice updates per second: every rank runs one replica of `nodes` nodes for `steps` steps."""
    return nodes * steps * ws / seconds / 1e9


KERNEL_SOURCES = ("paper_1904_11386_gb300/csrc/bulk_split.cu", "paper_1904_11386_gb300/csrc/pull.cuh",
                  "paper_1904_11386_gb300/csrc/async_copy.cuh", "paper_1904_11386_gb300/csrc/pdl.cuh",
                  "paper_1904_11386_gb300/csrc/scbb_internal.cuh")


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload_name: str):
    """DRAM bytes (read + write) per launch of the bulk kernel from the committed ncu summary of this
    workload, or None when there is none or the kernel source changed since it was taken."""
    import re

    path = os.path.join(ROOT, "profiles", f"bulk_{workload_name}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", txt)
    if not m_hash or not m_tr or m_hash.group(1) != kernel_source_hash():
        return None
    return int(m_tr.group(1))


def storage_beside(prob, args, ws, local, n_upd, peak, storage):
    """The same workload with the populations stored as FP16 or BF16 (FP32 arithmetic), timed the same way:
    K steps as the user call runs them, then K steps with events around every bulk launch."""
    import copy

    import torch

    from paper_1904_11386_gb300 import scbb

    p16 = copy.deepcopy(prob)
    p16.storage = STORAGE[storage]
    rhoA, rhoB = p16.initial_density()
    sim = scbb.Sim(p16, rhoA, rhoB, device=f"cuda:{local}")
    st = sim.stream
    sim.scbb_step(args.warmup)
    sim.scbb_sync()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sim.scbb_step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = replica_max(e0.elapsed_time(e1), ws, f"cuda:{local}")
    sim.scbb_enable_timing(True)
    sim.scbb_step(args.steps)
    bulk_ms, bulk_n = sim.scbb_kernel_time()
    sim.scbb_enable_timing(False)
    sim.scbb_sync()
    sim.close()
    bulk_s = bulk_ms / max(bulk_n, 1) / 1e3
    achieved = BYTES_PER_LU_16 * n_upd / bulk_s / 1e9
    return {"value": aggregate_glups(prob.n_nodes, args.steps, ws, ms / 1e3), "unit": "GLUPS",
            "ms_per_step": ms / args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_lu": BYTES_PER_LU_16, "kernel_ms": bulk_s * 1e3,
                         "traffic": recorded_traffic(f"{args.workload}-{storage}")},
            "error_vs_fp64_oracle": STORAGE_ERROR[storage]}


def _timed_batch(probs, args, dev, shared, clocks=None):
    """Steps a batch of fresh contexts of probs (warm-up, then args.steps timed on the batch stream); returns
    (ms, launches, shared bulk phase or not, clock record)."""
    import torch

    from paper_1904_11386_gb300 import scbb

    old = os.environ.get("SCBB_BATCH_PERSISTENT")
    os.environ["SCBB_BATCH_PERSISTENT"] = "1" if shared else "0"
    try:
        sims = [scbb.Sim(p, device=dev) for p in probs]
        batch = scbb.Batch(sims)
    finally:
        if old is None:
            del os.environ["SCBB_BATCH_PERSISTENT"]
        else:
            os.environ["SCBB_BATCH_PERSISTENT"] = old
    bst = batch.stream
    batch.scbb_batch_step(args.warmup)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    l0 = sum(s.scbb_launch_count() for s in sims)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bst)
    batch.scbb_batch_step(args.steps)
    e1.record(bst)
    torch.cuda.synchronize()
    launches = sum(s.scbb_launch_count() for s in sims) - l0
    clk = clocks.stop() if clocks else None
    for s in sims:
        s.scbb_sync()
    mode = batch.scbb_batch_shared_bulk()
    batch.close()
    for s in sims:
        s.close()
    return e0.elapsed_time(e1), launches, mode, clk


def run_batch(args, probs, label, ws, rank, local):
    """The sweep of independent boxes: steps of all boxes together, pairs of steps replayed from one CUDA graph
    with a branch per box (the library's default for bounce-back boxes), against the same batch with the bulk
    phase of every box in one persistent cooperative launch per step (the rest of each box's step on its own
    stream), and against the boxes stepped one after another on one stream, kernel by kernel (looping single
    launches).  value = lattice updates of all boxes per second of the default batched run."""
    import torch

    from paper_1904_11386_gb300 import scbb

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    nodes = sum(p.n_nodes for p in probs)
    n_upd = sum(p.nx * p.ny * (p.nz - 2 * p.walls) for p in probs)
    clocks = Clocks()
    ms, launches, _, clk = _timed_batch(probs, args, dev, False, clocks)
    ms = replica_max(ms, ws, dev)
    ms_sh, launches_sh, shared, _ = _timed_batch(probs, args, dev, True)
    ms_sh = replica_max(ms_sh, ws, dev)
    # looping single launches: all boxes on one stream, one box after another, one step per call
    one = torch.cuda.Stream(device=dev)
    loop_sims = [scbb.Sim(p, device=dev, stream=one) for p in probs]
    for s in loop_sims:
        s.scbb_step(args.warmup)
    torch.cuda.synchronize()
    k_loop = min(args.steps, 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(one)
    for _ in range(k_loop):
        for s in loop_sims:
            s.scbb_step(1)
    e1.record(one)
    torch.cuda.synchronize()
    ms_loop = replica_max(e0.elapsed_time(e1), ws, dev)
    for s in loop_sims:
        s.scbb_sync()
        s.close()
    peak, src = peak_hbm()
    # the boxes' bulk kernels overlap each other and the other kernels of the step, so per-launch events do not
    # give a kernel duration here: the bulk kernels' algorithmic bytes per batched step over the whole step
    # time bound their throughput from below
    achieved = BYTES_PER_LU * n_upd / (ms / args.steps / 1e3) / 1e9
    out = {"metric": "2-component D3Q19 lattice updates per second, full coupled step (GLUPS); batched sweep",
           "value": aggregate_glups(nodes, args.steps, ws, ms / 1e3), "unit": "GLUPS", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": label, "boxes": len(probs), "nodes": nodes, "parallelism": f"replicas x{ws}",
                      "l2": f"inputs larger than L2 (populations 2 x {2 * 19 * 4 * nodes / 1e6:.0f} MB)"},
           "shared_bulk_launch": {"value": aggregate_glups(nodes, args.steps, ws, ms_sh / 1e3), "unit": "GLUPS",
                                  "gpu_launches": launches_sh, "active": bool(shared),
                                  "how": "the bulk phase of all boxes in one persistent cooperative launch per "
                                         "step (kernel A, bounded grid barrier, kernel B), the rest per box"},
           "looped_single_launches": {"value": aggregate_glups(nodes, k_loop, ws, ms_loop / 1e3), "unit": "GLUPS",
                                      "steps": k_loop,
                                      "how": "all boxes on one stream, box after box, one step per call"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": None,
                        "kernel": "bulk phase of all boxes: algorithmic bytes per batched step / whole step time "
                                  "(a lower bound; the step also runs the bookkeeping kernels)",
                        "bytes_per_lu": BYTES_PER_LU, "units_per_step": n_upd, "peak_source": src},
           "gpu_launches": launches, "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(probs[0], args.cpu_seconds)
        out["cpu_baseline"]["sample"] += " (box 0 of the sweep)"
    return out


def cpu_baseline(prob, seconds=15.0):
    """The FP64 oracle as it stands, on this host's cores, on a bounded number of steps of the same workload."""
    from oracle import oracle as O

    s = O.OracleSim(prob)
    s.step(1)                                    # first touch
    n, t0 = 0, time.perf_counter()
    while True:
        s.step(1)
        n += 1
        dt = time.perf_counter() - t0
        if dt > seconds or n >= 200:
            break
    return {"value": prob.n_nodes * n / dt / 1e9, "unit": "GLUPS", "cores": O.threads(), "kind": "oracle",
            "sample": f"{n} full time steps of the {prob.nx}x{prob.ny}x{prob.nz} workload ({dt:.1f} s)"}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def run_reference_batch(args, probs, label, rank):
    """Reference arm of the sweep: the FP64 oracle steps every box in turn on the host cores."""
    if rank != 0:
        return
    from oracle import oracle as O

    sims = [O.OracleSim(p) for p in probs]
    for s in sims:
        s.step(args.warmup)
    t0 = time.perf_counter()
    for s in sims:
        s.step(args.steps)
    dt = time.perf_counter() - t0
    nodes = sum(p.n_nodes for p in probs)
    v = nodes * args.steps / dt / 1e9
    print(json.dumps({"metric": "2-component D3Q19 lattice updates per second, full coupled step (GLUPS); batched sweep",
                      "value": v, "unit": "GLUPS", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                      "config": {"workload": label, "boxes": len(probs), "nodes": nodes},
                      "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": O.threads(), "kind": "oracle",
                                       "sample": f"{args.steps} full time steps of every box"},
                      "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def run_adjoint(args, prob, label, ws, rank, local, n_steps=2000, every=100):
    """Forward (n steps with a checkpoint every `every` steps) and backward (recompute each segment, adjoint
    steps) of the adjoint, each timed with CUDA events on the context stream after a warm-up pair; value =
    backward time / forward time.  With a capsule the loss is its centre-of-mass height (the mean z of its
    vertices) and the gradients are those of scbb_adjoint_backward_capsule; without, the weighted centres of
    mass of the two components."""
    import numpy as np
    import torch

    from paper_1904_11386_gb300 import scbb

    torch.cuda.set_device(local)
    rhoA0, rhoB0 = prob.initial_density()
    z, _, x = np.meshgrid(np.arange(prob.nz), np.arange(prob.ny), np.arange(prob.nx), indexing="ij")
    wA, wB = z.astype(np.float64), 0.5 * x.astype(np.float64)
    sim = scbb.Sim(prob, rhoA0, rhoB0, device=f"cuda:{local}")
    shape = sim.scbb_autotune()              # a single 64^3 box fills the GPU only with short z-segments
    capsule = bool(prob.capsules)
    nv = int(sum(sim.nv))
    state0 = sim.scbb_save()                 # the initial state (populations and vertices) of both passes
    adj = scbb.Adjoint(sim, n_steps, every)
    st = sim.stream
    times = []
    for rep in range(2):                     # the first pair warms up
        sim.scbb_load(state0)
        sim.scbb_sync()
        l0 = sim.scbb_launch_count()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        adj.scbb_adjoint_forward()
        e1.record(st)
        if capsule:
            gX = np.zeros((nv, 3))
            gX[:, 2] = 1.0 / nv
            dmod, _, dG, dg = adj.scbb_adjoint_backward_capsule(gX)
        else:
            dG, dg, _, _ = adj.scbb_adjoint_backward(wA, wB)
        e2.record(st)
        torch.cuda.synchronize()
        times.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        launches = sim.scbb_launch_count() - l0
    fwd_ms, bwd_ms = times[-1]
    fwd_ms = replica_max(fwd_ms, ws, f"cuda:{local}")
    bwd_ms = replica_max(bwd_ms, ws, f"cuda:{local}")
    nodes = prob.n_nodes
    what = "capsule (immersed boundary) adjoint" if capsule else "fluid adjoint"
    out = {"metric": f"{what} backward / forward time ({n_steps} steps, checkpoint every {every})",
           "value": bwd_ms / fwd_ms, "unit": "x", "n_gpus": ws, "steps": n_steps, "warmup": 1,
           "ms_per_step": (fwd_ms + bwd_ms) / n_steps, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": label, "lattice": [prob.nx, prob.ny, prob.nz], "nodes": nodes,
                      "checkpoint_every": every, "bulk_shape": shape, "parallelism": f"replicas x{ws}"},
           "forward_ms": fwd_ms, "backward_ms": bwd_ms,
           "forward_glups": aggregate_glups(nodes, n_steps, ws, fwd_ms / 1e3),
           "adjoint_workspace_bytes": adj.nbytes, "context_workspace_bytes": int(sim.workspace.numel()),
           "gradients": {"dL_dG": dG, "dL_dg": list(map(float, dg))},
           "gradient_check": "tests/test_gpu_adjoint.py: FP64 central differences of the oracle, 32^3, 100 steps",
           "gpu_launches": launches}
    if capsule:
        out["gradients"].update({"dCOMz_dkS": float(dmod[0, 0]), "dCOMz_dkB": float(dmod[0, 1]),
                                 "dCOMz_dkV": float(dmod[0, 2])})
    adj.close()
    sim.close()
    return out


def run_reference(args, prob, label, ws, rank):
    """Reference arm: the FP64 oracle (plain C, OpenMP) on the host cores; each step one full time step."""
    if rank != 0:
        return
    from oracle import oracle as O

    s = O.OracleSim(prob)
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    v = prob.n_nodes * args.steps / dt / 1e9
    out = {"metric": METRIC, "value": v,
           "unit": "GLUPS", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": label, "lattice": [prob.nx, prob.ny, prob.nz]},
           "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": O.threads(), "kind": "oracle",
                            "sample": f"{args.steps} full time steps"},
           "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adsorb128")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="adsorb128: skip the batch48 and adjoint64 summaries of the default line")
    ap.add_argument("--no-fp16", action="store_true",
                    help="skip the 16-bit storage figures (FP16, BF16) beside the FP32 ones")
    ap.add_argument("--adj-steps", type=int, default=2000, help="adjoint64: steps differentiated")
    ap.add_argument("--adj-every", type=int, default=100, help="adjoint64: steps between checkpoints")
    ap.add_argument("--storage", default="fp32", choices=list(STORAGE),
                    help="population storage on the GPU (arithmetic is FP32 either way)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_setup()
    prob, label = workload(args.workload)
    if args.workload in ("adjoint64", "adjoint64-fluid") and args.impl == "ours":
        out = run_adjoint(args, prob, label, ws, rank, local, n_steps=args.adj_steps, every=args.adj_every)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return
    if args.workload == "batch48":
        if args.impl == "reference":
            run_reference_batch(args, prob, label, rank)
        else:
            out = run_batch(args, prob, label, ws, rank, local)
            if rank == 0:
                print(json.dumps(out), flush=True)
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return
    if args.storage != "fp32":
        prob.storage = STORAGE[args.storage]
        label += f"; populations stored as {args.storage.upper()}"
    if args.impl == "reference":
        run_reference(args, prob, label, ws, rank)
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    from paper_1904_11386_gb300 import scbb

    torch.cuda.set_device(local)
    rhoA, rhoB = prob.initial_density()
    sim = scbb.Sim(prob, rhoA, rhoB, device=f"cuda:{local}")
    st = sim.stream
    sim.scbb_step(args.warmup)
    sim.scbb_sync()

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-resident timing of K full steps, run as a user's scbb_step runs them (pairs of steps replayed
    # from a captured CUDA graph)
    clocks = Clocks()
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = sim.scbb_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sim.scbb_step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    launches = sim.scbb_launch_count() - l0
    ms = e0.elapsed_time(e1)
    # ---- the bulk kernel's launch durations: K more steps with a pair of CUDA events around every bulk launch
    # on the context stream (timed steps launch kernel by kernel)
    sim.scbb_enable_timing(True)
    torch.cuda.synchronize()
    sim.scbb_step(args.steps)
    bulk_ms, bulk_n = sim.scbb_kernel_time()
    sim.scbb_enable_timing(False)
    sim.scbb_sync()
    clk = clocks.stop()
    ms = replica_max(ms, ws, f"cuda:{local}")
    N = prob.n_nodes
    value = aggregate_glups(N, args.steps, ws, ms / 1e3)

    # ---- end to end through the C ABI with host buffers in pinned memory: upload the initial fields (FP64),
    # K steps, read the fields back (FP64)
    def pinned(n):
        return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()

    hA, hB = pinned(N), pinned(N)
    hA[:] = rhoA.ravel()
    hB[:] = rhoB.ravel()
    out = (pinned(N), pinned(N), pinned(3 * N))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.scbb_set_density(hA, hB)
    sim.scbb_step(args.steps)
    a, b, u = sim.scbb_get_fields(out=out)
    e2e_s = replica_max(time.perf_counter() - t0, ws, f"cuda:{local}")
    if not np.isfinite(a).all():
        raise SystemExit("non-finite densities")
    h2d = hA.nbytes + hB.nbytes
    d2h = sum(o.nbytes for o in out)
    e2e = {"value": aggregate_glups(N, args.steps, ws, e2e_s), "unit": "GLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "job": f"set_density (pinned host FP64 rho^A, rho^B) + {args.steps} steps + get_fields (pinned host "
                  f"FP64 rho^A, rho^B, u)"}

    peak, src = peak_hbm()
    bulk_avg_s = bulk_ms / max(bulk_n, 1) / 1e3
    n_upd = prob.nx * prob.ny * (prob.nz - 2 * prob.walls)    # nodes one bulk launch updates (no wall planes)
    bpl = bytes_per_lu(args.storage)
    achieved = bpl * n_upd / bulk_avg_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(args.workload + ("" if args.storage == "fp32" else "-" + args.storage)),
            "kernel": "bulk phase: k_moments_staged (stream, moments) + k_collide_pair (Shan-Chen force, collide)",
            "bytes_per_lu": bpl, "units_per_launch": n_upd, "peak_source": src,
            "kernel_ms": bulk_avg_s * 1e3, "kernel_share": bulk_avg_s * 1e3 / (ms / args.steps) if ms > 0 else None,
            "kernel_timing": f"{bulk_n} bulk launches bracketed by CUDA events (second region of {args.steps} steps)"}

    out = {"metric": METRIC,
           "value": value, "unit": "GLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": label, "lattice": [prob.nx, prob.ny, prob.nz], "nodes": N,
                      "vertices": int(sum(sim.nv)), "parallelism": f"replicas x{ws}",
                      "storage": args.storage,
                      "l2": f"inputs larger than L2 (populations {2 * 19 * N * (4 if args.storage == 'fp32' else 2) / 1e6:.0f} MB a lattice)"},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    nv = int(sum(sim.nv))
    if nv:
        # membrane vertices moved per second by the whole job (the same timed region as value)
        out["vertex_updates_per_s"] = nv * args.steps * ws / (ms / 1e3)
    sim.close()
    if args.storage == "fp32" and not args.no_fp16:
        for st16 in ("fp16", "bf16"):
            out[f"{st16}_storage"] = storage_beside(prob, args, ws, local, n_upd, peak, st16)
    if args.workload == "adsorb128" and args.storage == "fp32" and not args.no_extras:
        # the batched and differentiated forms, measured in the same run (their own workloads)
        bprobs, blabel = workload("batch48")
        bargs = argparse.Namespace(**{**vars(args), "no_cpu_baseline": True})
        b = run_batch(bargs, bprobs, blabel, ws, rank, local)
        out["batch48"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "shared_bulk_launch",
                                            "looped_single_launches", "gpu_launches")}
        out["batch48"]["workload"] = blabel
        aprob, alabel = workload("adjoint64")
        a = run_adjoint(args, aprob, alabel, ws, rank, local, n_steps=args.adj_steps, every=args.adj_every)
        out["adjoint64"] = {k: a[k] for k in ("value", "unit", "forward_ms", "backward_ms", "forward_glups",
                                              "adjoint_workspace_bytes", "gpu_launches")}
        out["adjoint64"]["metric"] = a["metric"]
        out["adjoint64"]["workload"] = alabel
        fprob, flabel = workload("adjoint64-fluid")
        f = run_adjoint(args, fprob, flabel, ws, rank, local, n_steps=args.adj_steps, every=args.adj_every)
        out["adjoint64"]["fluid_only"] = {k: f[k] for k in ("value", "unit", "forward_ms", "backward_ms",
                                                            "adjoint_workspace_bytes", "gpu_launches", "metric")}
        out["adjoint64"]["fluid_only"]["workload"] = flabel
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
