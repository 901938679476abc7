"""Benchmark of the LBE time step (MLUPS and fraction of the HBM roofline).

One "step" is one full LBE time step of the lattice: the fused link-flux +
collide-stream sweep, the advection sweep and the Poisson solve to tolerance
(the induced charge is read through the e2e path).  Default workload: the
64x64x256 electro-osmosis lattice (plates at z = 0 and z = 255, voltage 0.2,
tangential field 1e-3, Debye length 16, l_B = 1.44, tau = 1), from the
uncharged capacitor with the voltage applied.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload eof|coax|plates|porous] [--precision fp64]
                    [--batch-steps K2]

Beside the main workload the line carries a "batched" object: the batched
FP32 form on the 256-instance sweep of parallel-plate and coaxial capacitors
(seeded sizes, Debye lengths and voltages), timed as one graph launch per
step, with the plain FP64 single-lattice form timed on a sample of the same
instances for comparison.

Under torchrun (N > 1) every rank advances its own replica of the lattice
(the workload does not shard across GPUs in this build); ``value`` sums the
lattice updates of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1907_04732_gb300 import workloads as wl  # noqa: E402

METRIC = "MLUPS"
UNIT = "MLUPS"


def make_workload(name: str):
    if name == "eof":
        return wl.eof_plates()
    if name == "coax":
        return wl.coax_capacitor()
    if name == "plates":
        return wl.plate_capacitor()
    if name == "porous":
        return wl.porous_electrode()
    raise SystemExit(f"unknown workload {name}")


def section(w, side=16):
    """Periodic x-y section of a translation-invariant workload (the oracle's
    bounded sample); None if the workload is not invariant along x and y."""
    if w.name.startswith(("eof_", "plates_")):
        nx, ny, nz = w.shape
        ids = w.ids[:, :min(side, ny), :min(side, nx)].copy()
        return w.with_(ids=ids, name=w.name + f"_section{ids.shape[2]}x{ids.shape[1]}")
    return None


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value of x over the ranks (the slowest rank's time); the
    process group is NCCL on the GPU box (device "cuda"), gloo in the CPU
    tests (device "cpu")."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, nodes_per_rank: int, steps: int, seconds: float) -> float:
    """Lattice updates of all ranks (one replica each) over the slowest
    rank's time."""
    return world * nodes_per_rank * steps / seconds / 1e6


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic bytes per fluid node (the method's own data, each element read
# or written once; neighbour re-reads come from cache).  The fused sweep of
# the FP32 deviation form moves 19 populations in and out (152 B), the two
# solute amounts (16 B at 32 bits each), the potential (4 B), the geometry
# (1 B) and writes the velocity for the advection (12 B): 185 B.  The
# implementation moves more (64-bit solute amounts, a 16 B velocity record,
# the link records of the prep kernel): IMPL_BYTES.
BYTES = {}
BYTES["fp64"] = {
    # 19 populations read + 19 written, n_k read + n*_k written, phi read,
    # u written (3), geometry
    "sweep": lambda ns: 8 * (19 + 19 + 2 * ns + 1 + 3) + 1,
    # n*_k read, n_k written, u read (3)
    "advect": lambda ns: 8 * (2 * ns + 3),
    # one Jacobi-preconditioned CG iteration: matvec (p read, q write),
    # update (phi, res, p, q read; phi, res write), direction (res, p read;
    # p write)
    "cg_iter": lambda ns: 8 * (2 + 6 + 3),
}
BYTES["fp32"] = {
    "sweep": lambda ns: 4 * (19 + 19) + 4 * 2 * ns + 4 + 1 + 4 * 3,
    # solute read and written (32 bits each), velocity read (3 x 4 B)
    "advect": lambda ns: 4 * 2 * ns + 4 * 3,
    # one multigrid-preconditioned CG iteration, level 0 (4 B vectors):
    # update (u, p, w, s, x, r read; p, s, x, r, u written: 44 B),
    # restriction (r, u: 8 B), prolongation (u read, t written: 8 B),
    # post-smoothing (r, t read, u written: 12 B), stencil and dot products
    # (u, r read, w written: 12 B) = 84 B; coarse levels (27-point operator,
    # 1/8 of the nodes per level): about 16 B per fine node
    "cg_iter": lambda ns: 84 + 16,
}
IMPL_BYTES = {
    # prep (mask, potential, two 64-bit amounts read; 16 B record written) +
    # sweep (populations, record, mask, amounts read and written, 16 B
    # velocity record)
    "fp32": {"sweep": lambda ns: (4 + 4 + 16 + 16) + (152 + 16 + 4 + 32 + 16),
             "advect": lambda ns: 32 + 16 + 8 * 8 + 8},
}

# DRAM bytes per launch of the fused sweep from an ncu capture, valid only
# for the kernel source it was taken from (a hash of the sweep's sources)
SWEEP_TRAFFIC = {
    # k_prep32 + k_sweep32 (odd in-place step), one launch each, from an ncu
    # --set full capture of these sources on GB300: 20.974592 + 116.611328 MB
    # read, 53.602816 MB written
    ("fp32", "eof_64x64x256", "c615e5a71457a79a"): 191188736,
}


def sweep_source_hash() -> str:
    import hashlib
    hsh = hashlib.sha256()
    for f in ("fp32_device.cuh", "kernels_fp32.cu", "lbe_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1907_04732_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_lattice(w, tol):
    from oracle import Oracle
    o = Oracle(w.shape, w.periodic, tau=w.tau, bjerrum=w.bjerrum, z=w.z, D=w.D, rho_bulk=w.rho_bulk,
               e_app=w.e_app, flow=w.flow, tol=tol)
    o.set_geometry(w.ids, w.n_elec)
    o.set_voltage(w.psi)
    return o


def cpu_baseline(w, tol, budget_s=15.0):
    """Time the FP64 oracle, as it stands, on a bounded sample of the
    workload: a 16x16 periodic section (or the full lattice when not
    translation invariant), warm-started from its initial state."""
    sub = section(w) or w
    o = oracle_lattice(sub, tol)
    o.init()
    o.step(1)  # first step outside the timing (page-in)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", 0)) or os.cpu_count()
    return {"value": sub.nodes * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{steps} FP64 oracle steps of the {sub.shape[0]}x{sub.shape[1]}x{sub.shape[2]} "
                      f"periodic section of {w.name} after its init ({dt:.1f} s, OpenMP)"}


def cpu_baseline_child(workload: str, tol, budget_s, threads=None):
    """cpu_baseline in a child process (the GPU process never loads the
    oracle), on all host cores or on `threads` threads; None if it fails."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline(bench.make_workload(%r), %r, %r)))"
            % (ROOT, workload, tol, budget_s))
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    try:
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=120 + 4 * budget_s)
        return json.loads(p.stdout.strip().splitlines()[-1]) if p.returncode == 0 else None
    except Exception:
        return None


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the
    implementer and part codes), with the machine type."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                k, v = k.strip(), v.strip()
                if k in ("model name", "CPU implementer", "CPU part") and k not in fields:
                    fields[k] = v
    except OSError:
        pass
    name = fields.get("model name") or " ".join(f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part")
                                                if k in fields)
    return f"{platform.machine()} {name}".strip()


def run_reference(args, w):
    """Reference arm: the plain FP64 oracle (CPU) on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sub = section(w) or w
    o = oracle_lattice(sub, args.tol)
    o.init()
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", 0)) or os.cpu_count()
    val = sub.nodes * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "sample": sub.name},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps of the {sub.shape} section of {w.name}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_leg(args, lbe, torch, stream, peak):
    """The batched FP32 form on the 256-instance capacitor sweep: MLUPS of
    one graph launch per step over all instances, the fused sweep's HBM
    fraction, and the plain FP64 form timed instance by instance on a
    sample (largest, smallest and four seeded others)."""
    import numpy as np
    ws = wl.batch_instances(256)
    b = lbe.Batch(ws, tol=args.tol, stream=stream.cuda_stream)
    b.init()
    grid, tuned = b.tuning()
    for _ in range(args.batch_warmup):
        b.step(1)
    torch.cuda.synchronize()
    nodes = sum(w.nodes for w in ws)
    fluid = sum(int((w.ids == 0).sum()) for w in ws)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(args.batch_steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.batch_steps
    st = b.stats()
    b.profile_begin()
    b.step(2)
    prof = b.profile_end()
    q = b.charge()
    b.close()
    sweep_ms = prof.sweep_ms / max(prof.sweep_launches, 1)
    sweep_gbs = BYTES["fp32"]["sweep"](2) * fluid / (sweep_ms * 1e-3) / 1e9
    # plain FP64 single-lattice form on a sample of the instances
    rng = np.random.Generator(np.random.PCG64(wl.SEED))
    sizes = [w.nodes for w in ws]
    sample = sorted({int(np.argmax(sizes)), int(np.argmin(sizes))} |
                    set(int(i) for i in rng.choice(len(ws), 4, replace=False)))
    if args.compare_steps == 0:
        sample = []
    t64, n64 = 0.0, 0
    for i in sample:
        w = ws[i]
        lat = lbe.Lattice(lbe.params_for(w, tol=args.tol, precision=lbe.LBE_FP64), stream=stream.cuda_stream)
        lat.set_geometry(w.ids, w.n_elec)
        lat.set_voltage(w.psi)
        lat.init()
        lat.step(2)
        torch.cuda.synchronize()
        ev0.record(stream)
        lat.step(3)
        ev1.record(stream)
        torch.cuda.synchronize()
        t64 += ev0.elapsed_time(ev1) / 3
        n64 += w.nodes
        lat.close()
    fp64_mlups = n64 / (t64 * 1e-3) / 1e6 if sample else None
    value = nodes / (ms * 1e-3) / 1e6
    return {"workload": "256 plate/coax capacitors (seeded gaps 32-512, sides 8-64, Debye 2-32, "
                        "voltages -0.5..0.5)",
            "instances": len(ws), "nodes": nodes, "fluid_nodes": fluid,
            "value": value, "unit": UNIT, "ms_per_step": ms, "steps": args.batch_steps,
            "launch": "one CUDA graph launch per step (persistent kernels over all instances)",
            "autotuned_grid_blocks": grid, "tuned_sweep_ms": tuned,
            "phases_ms": {"sweep": sweep_ms,
                          "advect": prof.advect_ms / max(prof.advect_launches, 1),
                          "poisson": prof.poisson_ms / max(prof.sweep_launches, 1)},
            "sweep_roofline": {"kernel": "kb_sweep (batched fused sweep)", "bound": "hbm",
                               "achieved": sweep_gbs, "peak": peak, "unit": "GB/s", "frac": sweep_gbs / peak},
            "cg_iters_per_step_summed_over_instances": st.poisson_iters / max(st.poisson_solves, 1),
            "cg_iters_per_step_max_instance": st.poisson_max_iters,
            "fp64_plain": {"value": fp64_mlups, "unit": UNIT,
                           "speedup_batched_fp32": value / fp64_mlups if fp64_mlups else None,
                           "sample": f"instances {sample}, one lattice at a time, 3 timed steps each"},
            "charge_finite": bool(np.all(np.isfinite(q)))}


def adjoint_leg(args, lbe, torch, stream):
    """Gradient of the induced charge after T steps on the 256x256x128
    porous electrode (solvent at rest): FP32 forward with checkpoints placed
    by the binomial (revolve) schedule within a device-memory budget (or
    every K steps with --adjoint-every), then the reverse sweep
    (recomputation, adjoint Poisson solves), timed with CUDA events; the
    plain FP64 forward step on the same lattice for comparison."""
    import numpy as np
    w = wl.porous_electrode()
    p = lbe.params_for(w, tol=args.tol, precision=lbe.LBE_FP32)
    lat = lbe.Lattice(p, stream=stream.cuda_stream)
    lat.set_geometry(w.ids, w.n_elec)
    lat.set_voltage(w.psi)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    per_slot = 48 * w.nodes  # solute (2 x 8 B), potential and its 3 earlier values (FP64)
    if args.adjoint_every > 0:
        q = lat.adjoint_forward(args.adjoint_steps, args.adjoint_every)
        slots = -(-args.adjoint_steps // args.adjoint_every) + 1
        ck_bytes, seg_bytes = slots * per_slot, args.adjoint_every * 20 * w.nodes
        schedule = "uniform, every %d steps" % args.adjoint_every
    else:
        budget = int(args.adjoint_budget_gb * 1e9)
        q = lat.adjoint_forward_budget(args.adjoint_steps, budget)
        slots = min(budget // per_slot, args.adjoint_steps + 2)
        ck_bytes, seg_bytes = slots * per_slot, 0
        schedule = "binomial (revolve), %d slots within %.1f GB" % (slots, args.adjoint_budget_gb)
    ev[1].record(stream)
    g, dchi = lat.adjoint_backward([1.0, 0.0], 1)
    ev[2].record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    lat.close()
    T = args.adjoint_steps
    # plain FP64 forward on the same lattice
    ms64 = None
    if args.compare_steps > 0:
        p64 = lbe.params_for(w, tol=args.tol, precision=lbe.LBE_FP64)
        l64 = lbe.Lattice(p64, stream=stream.cuda_stream)
        l64.set_geometry(w.ids, w.n_elec)
        l64.set_voltage(w.psi)
        l64.init()
        l64.step(3)
        torch.cuda.synchronize()
        ev[0].record(stream)
        l64.step(5)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms64 = ev[0].elapsed_time(ev[1]) / 5
        l64.close()
    node_steps = w.nodes * T
    return {"workload": w.name + " (200 seeded spheres r 6-12 on a backing plate, counter plate; flow off)",
            "objective": "Q_1 after T steps", "steps": T, "checkpoint_schedule": schedule,
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "forward_mlups": node_steps / (fwd_ms * 1e-3) / 1e6,
            "gradient_mlups": node_steps / ((fwd_ms + bwd_ms) * 1e-3) / 1e6,
            "backward_over_forward": bwd_ms / fwd_ms,
            "recomputed_steps": int(g.recomputed_steps), "adjoint_cg_iters": int(g.poisson_iters),
            "backward_phases_ms": {"recompute": g.recompute_ms, "flux_transpose": g.flux_ms,
                                   "adjoint_solves": g.solve_ms},
            "checkpoint_bytes": ck_bytes, "segment_bytes": seg_bytes,
            "recomputed_per_step": g.recomputed_steps / max(T, 1),
            "Q": [float(v) for v in q], "dQ1_dpsi": [float(v) for v in g.dpsi[:2]],
            "dQ1_drho_bulk": float(g.drho_bulk), "dQ1_dD": [float(v) for v in g.dD[:2]],
            "dQ1_dchi_absmax": float(np.abs(dchi).max()),
            "fp64_plain_forward": None if ms64 is None else {
                "ms_per_step": ms64, "value": w.nodes / (ms64 * 1e-3) / 1e6, "unit": UNIT,
                "gradient_vs_fp64_forward_time": (fwd_ms + bwd_ms) / (ms64 * T)}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="eof")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--compare-steps", type=int, default=5,
                    help="steps of the plain FP64 form timed for comparison (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="timed steps of the 256-instance batched form (0 = skip)")
    ap.add_argument("--batch-warmup", type=int, default=3)
    ap.add_argument("--adjoint-steps", type=int, default=2000,
                    help="steps of the porous-electrode gradient run (0 = skip)")
    ap.add_argument("--adjoint-every", type=int, default=0,
                    help="uniform checkpoints every K steps (0: the binomial schedule within --adjoint-budget-gb)")
    ap.add_argument("--adjoint-budget-gb", type=float, default=8.0)
    args = ap.parse_args()
    w = make_workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w)
        return

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1907_04732_gb300 import build as nvbuild
    from paper_1907_04732_gb300 import lbe
    nvbuild.build()
    lbe.load()

    stream = torch.cuda.Stream()
    prec = lbe.LBE_FP32 if args.precision == "fp32" else lbe.LBE_FP64
    params = lbe.params_for(w, tol=args.tol, precision=prec)
    lat = lbe.Lattice(params, stream=stream.cuda_stream)
    lat.set_geometry(w.ids, w.n_elec)
    lat.set_voltage(w.psi)
    lat.init()
    fluid = int((w.ids == 0).sum())

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        lat.step(1)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.profile_begin()
    ev0.record(stream)
    lat.step(args.steps)  # K steps in one call: no host round trip between steps
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = lat.profile_end()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms / args.steps
    value = whole_job_mlups(world, w.nodes, args.steps, ms * 1e-3)

    # e2e through the public API with host buffers: per step the electrode
    # potentials go host->device, the induced charges device->host
    psi = np.asarray(w.psi, dtype=np.float64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        lat.set_voltage(psi)
        lat.step(1)
        q = lat.charge()
    torch.cuda.synchronize()
    e2e_dt = max_over_ranks(time.perf_counter() - t0, world)
    e2e_val = whole_job_mlups(world, w.nodes, args.e2e_steps, e2e_dt)

    peak, peak_kind = load_peaks()
    ns = len(w.z)
    B = BYTES[args.precision]
    iters = prof.poisson_iters / max(prof.poisson_solves, 1)
    phases = {"sweep": prof.sweep_ms / max(prof.sweep_launches, 1),
              "advect": prof.advect_ms / max(prof.advect_launches, 1),
              "poisson": prof.poisson_ms / max(prof.poisson_solves, 1)}
    sweep_bytes = B["sweep"](ns) * fluid
    sweep_gbs = sweep_bytes / (phases["sweep"] * 1e-3) / 1e9
    adv_bytes = B["advect"](ns) * fluid if w.flow else 0
    pois_bytes = B["cg_iter"](ns) * iters * fluid
    step_ms = ms_step
    shares = {k: v / step_ms for k, v in phases.items()}
    # The fused LBE sweep (its prep kernel included) is the kernel the HBM
    # roofline is reported for: algorithmic bytes / live CUDA-event time.
    traffic = SWEEP_TRAFFIC.get((args.precision, w.name, sweep_source_hash()))
    roof = {"kernel": "k_prep32 + k_sweep32 (fused link flux + force + BGK/Guo collide + stream)"
            if args.precision == "fp32" else "k_sweep (FP64 fused sweep)",
            "bound": "hbm", "achieved": sweep_gbs, "peak": peak, "unit": "GB/s", "frac": sweep_gbs / peak,
            "traffic": traffic,
            "bytes_per_node": B["sweep"](ns), "units_per_launch": fluid,
            "impl_bytes_per_node": IMPL_BYTES.get(args.precision, B)["sweep"](ns),
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "share_of_step": shares["sweep"]}
    step_bytes = sweep_bytes + adv_bytes + pois_bytes
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "value_fluid_nodes": whole_job_mlups(world, fluid, args.steps, ms * 1e-3),
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": w.name, "lattice": list(w.shape), "nodes": w.nodes, "fluid_nodes": fluid,
                   "precision": args.precision, "poisson_tol": args.tol,
                   "l2": ("inputs larger than L2 (129 MB): the sweep alone touches %.0f MB (populations "
                          "%s %.0f MB, link records, solute in and out, velocity records, mask)"
                          % (w.nodes * ((19 * 4 + 16 + 32 + 16 + 4) if args.precision == "fp32"
                                        else (19 * 8 * 2 + 8 + 32 + 24 + 4)) / 1e6,
                             "in place" if args.precision == "fp32" else "two buffers",
                             w.nodes * 19 * (4 if args.precision == "fp32" else 16) / 1e6)),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "phases_ms": phases, "phase_shares": shares,
        "poisson": {"ms_per_step": phases["poisson"], "cg_iters_per_step": iters,
                    "bytes_per_node_per_cg_iter": B["cg_iter"](ns),
                    "gbs": pois_bytes / (phases["poisson"] * 1e-3) / 1e9,
                    "hbm_frac": pois_bytes / (phases["poisson"] * 1e-3) / 1e9 / peak,
                    "note": ("refinement on the fixed-point potential (exact integer Laplacian, float-float "
                             "charge term), multigrid-preconditioned FP32 CG, cubic warm start in time; one CUDA "
                             "graph launch per solve (conditional while nodes for the refinement and CG loops); "
                             "its vectors stay in L2, so the fraction is of effective bandwidth")
                            if args.precision == "fp32" else
                            ("FP64 Jacobi-preconditioned CG in one CUDA graph launch per solve, cubic warm start "
                             "in time")},
        "step": {"bytes_per_node": step_bytes / fluid, "gbs": step_bytes / (step_ms * 1e-3) / 1e9,
                 "hbm_frac": step_bytes / (step_ms * 1e-3) / 1e9 / peak,
                 "parts": "fused sweep + advection + Poisson CG iterations (algorithmic bytes)"},
        "lb_part_hbm_frac": (sweep_bytes + adv_bytes) / ((phases["sweep"] + phases["advect"]) * 1e-3) / 1e9 / peak,
        "advect_gbs": adv_bytes / (phases["advect"] * 1e-3) / 1e9 if phases["advect"] > 0 else None,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * w.n_elec,
                "d2h_bytes_per_step": 8 * w.n_elec},
        "gpu_launches": int(prof.kernel_launches),
        "clocks": clk,
    }
    lat.close()
    if args.precision == "fp32" and args.compare_steps > 0:
        # the plain FP64 form on the same workload, same tolerance
        p64 = lbe.params_for(w, tol=args.tol, precision=lbe.LBE_FP64)
        l64 = lbe.Lattice(p64, stream=stream.cuda_stream)
        l64.set_geometry(w.ids, w.n_elec)
        l64.set_voltage(w.psi)
        l64.init()
        for _ in range(args.warmup):
            l64.step(1)
        torch.cuda.synchronize()
        ev0.record(stream)
        l64.step(args.compare_steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1) / args.compare_steps
        line["fp64_plain"] = {"value": w.nodes / (ms64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms64,
                              "steps": args.compare_steps, "speedup_fp32": ms64 / ms_step}
        l64.close()
    if args.batch_steps > 0:
        line["batched"] = batch_leg(args, lbe, torch, stream, peak)
    if args.adjoint_steps > 0:
        line["adjoint"] = adjoint_leg(args, lbe, torch, stream)
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline_child(args.workload, args.tol, 15.0)
        if cb is not None:
            one = cpu_baseline_child(args.workload, args.tol, 5.0, threads=1)
            cb["single_thread_value"] = one["value"] if one else None
            cb["process"] = "child processes (the GPU process does not load the oracle)"
        line["cpu_baseline"] = cb
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
