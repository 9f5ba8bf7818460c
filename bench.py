#!/usr/bin/env python
"""Throughput of the entanglement-aware MPS two-site update on GB300.

Workload (one "step"): a full 100-qubit brickwork circuit of depth 30 of
Haar-random SU(4) nearest-neighbour gates (seeded, synthetic), simulated from
|0...0> by the EA-MPS hot path: centre move, theta contraction, Jacobi SVD,
bond selection against the per-truncation fidelity target (global schedule,
F_min = 0.9) with a bond cap, and write-back.  The metric is two-qubit updates
per second over the whole circuit.

Arms
----
default           the CUDA path; ``value`` with the circuit resident in HBM,
                  ``e2e`` through the host-buffer C-ABI call (gates copied
                  host -> device with every launch, the chosen bond read back
                  after every gate, the inferred fidelity read back per step).
--impl reference  the FP64 CPU oracle (textbook MPS with LAPACK SVD) on the
                  host cores, on a bounded sample of the same circuit.

Multi-GPU: replicas only (the gates of one circuit form a single sequential
chain through the orthogonality centre); each rank runs its own circuit and
``value`` is the sum of updates over all ranks divided by the slowest rank's
time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-qubits", type=int, default=100)
    ap.add_argument("--depth", type=int, default=30)
    ap.add_argument("--f-min", type=float, default=0.9)
    ap.add_argument("--chi-cap", type=int, default=256)
    ap.add_argument("--fixed-chi", type=int, default=0)
    ap.add_argument("--seed", type=int, default=1002)
    ap.add_argument("--precision", default="tf32x3", choices=["tf32x3", "fp32", "fp64"])
    ap.add_argument("--svd-kernel", default="auto", choices=["auto", "tournament", "tournament-unsplit", "gram"],
                    help="layout of the Jacobi SVD (mps_options.svd_kernel)")
    ap.add_argument("--qr", default="both", choices=["moves", "precondition", "both", "none"],
                    help="Householder QR use (mps_options.qr): centre moves, the preconditioned gate SVD, "
                         "both, or neither (Jacobi orthogonalisation)")
    ap.add_argument("--cpu-sample-s", type=float, default=20.0, help="seconds of oracle work per CPU sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-target, chi = 512 and precision blocks of the bench line")
    ap.add_argument("--flush-mb", type=int, default=512, help="L2 flush buffer written between timed steps")
    ap.add_argument("--study", default="",
                    choices=["", "ttf", "mpo", "batch", "strategies", "grad", "vidal", "precision", "e1"],
                    help="ttf: time to target fidelity, EA against fixed bond dimensions; "
                         "mpo: the noisy EA-MPO workload (d = 4); "
                         "batch: 64 independent circuits run concurrently; "
                         "strategies: inferred vs true fidelity of the naive/global/nearest schedules; "
                         "grad: parameter-shift gradients of the layered ansatz as one batch; "
                         "vidal: the Vidal/Hastings form against the canonical update; "
                         "precision: tf32x3 / fp32 runs and the differentiable form against FP64 on the GPU")
    ap.add_argument("--micro-moves", action="store_true",
                    help="with --micro: shift the gate right by two sites each update, so that every update "
                         "also moves the orthogonality centre (a QR of a (2 CHI) x CHI site)")
    ap.add_argument("--micro", type=int, default=0, metavar="CHI",
                    help="instead of the circuit: a few two-site updates on a random canonical 24-site MPS "
                         "with every bond CHI (the launch configuration of the circuit's saturated gates)")
    return ap.parse_args(argv)


def bench_config(a, n_2q: int, world: int) -> dict:
    """The workload keys both arms print (the GPU arm and the oracle arm measure the same circuit)."""
    return {"workload": workload_name(a), "n_qubits": a.n_qubits, "depth": a.depth, "n_2q": n_2q, "seed": a.seed,
            "chi_cap": a.chi_cap, "f_min": a.f_min, "fixed_chi": a.fixed_chi, "strategy": "global",
            "l2": f"GPU arm: flushed between timed steps ({a.flush_mb} MB write); CPU arm: not applicable",
            "parallelism": "replicas" if world > 1 else "single"}


def workload_name(a) -> str:
    mode = f"fixed chi={a.fixed_chi}" if a.fixed_chi else f"EA F_min={a.f_min} global, chi cap {a.chi_cap}"
    return f"EA-MPS pure state, {a.n_qubits}-qubit chain, brickwork depth {a.depth}, Haar SU(4), {mode}"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max_sum(t_local: float, n_local: float, world: int, backend_device=None):
    """Max of the per-rank times and sum of the per-rank work (the replica aggregation)."""
    if world <= 1:
        return t_local, n_local
    import torch
    import torch.distributed as dist
    dev = backend_device if backend_device is not None else torch.device("cpu")
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    n = torch.tensor([n_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle sample
def cpu_oracle_sample(circ, a, seconds: float) -> dict:
    """Time the FP64 oracle on the first gates of the same circuit, bounded by ``seconds``."""
    from oracle import textbook_mps as T
    m = T.TextbookMPS(circ.n_qubits, f_min=a.f_min, n_2q=circ.n_2q, strategy=T.GLOBAL,
                      chi_max=a.chi_cap if not a.fixed_chi else 0, fixed_chi=a.fixed_chi)
    t0 = time.perf_counter()
    done = 0
    for q, u in circ.gates():
        m.apply_2q(q, u)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
    cores = int(threads) if threads else (os.cpu_count() or 1)
    return {"value": done / dt, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": f"first {done} of {circ.n_2q} gates of the same circuit from |0...0> "
                      f"({dt:.1f} s, NumPy/LAPACK FP64, max bond {max(m.bond_dims())}); early gates have "
                      f"smaller bonds, so this overstates the oracle's whole-circuit rate"}


def run_reference(a) -> int:
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    circ = W.brickwork_circuit(a.n_qubits, a.depth, a.seed)
    per_step = max(5.0, min(a.cpu_sample_s, 60.0))
    for _ in range(a.warmup):
        cpu_oracle_sample(circ, a, per_step / 4)
    vals, samples = [], []
    t_all = 0.0
    for _ in range(a.steps):
        r = cpu_oracle_sample(circ, a, per_step)
        vals.append(r["value"])
        samples.append(r)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "2-qubit MPS updates/s", "value": value, "unit": "updates/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "precision": "fp64", "config": bench_config(a, circ.n_2q, 1),
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": samples[-1]["cores"], "kind": "oracle",
                             "sample": samples[-1]["sample"]},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
# DRAM traffic of one theta 512 x 512 launch of the point-to-point Jacobi kernel, from the ncu
# capture named here (re-taken whenever that kernel changes; None when no capture of the current
# kernel exists)
TRAFFIC_512 = 2141184 + 34816
TRAFFIC_SOURCE = ("dram__bytes_read.sum + dram__bytes_write.sum of jacobi_kernel3<float, 16, 16, 1, 2> (the "
                  "row-split variant) in an ncu capture of bench.py --micro 256 --svd-kernel tournament "
                  "(profiles/jacobi_kernel3_theta512x512.md); not measured by this run")


def measured_peaks() -> dict:
    """The generated peaks of this GPU pool (HBM copy GB/s, bf16 TFLOP/s), if present."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def run_ours(a) -> int:
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2307_16870_gb300 as E
    prec = {"tf32x3": E.TF32X3, "fp32": E.FP32, "fp64": E.FP64}[a.precision]
    circ = W.brickwork_circuit(a.n_qubits, a.depth, a.seed + rank)
    n = circ.n_2q
    ops = circ.ops_array()                                        # (n, 4, 4) complex128
    ops_dev = torch.from_numpy(ops.view(np.float64).reshape(n, 32).copy()).to(dev)
    qs = np.asarray(circ.qs, dtype=np.int32)
    stream = torch.cuda.current_stream(dev)
    m = E.MPS(a.n_qubits, f_min=a.f_min, n_2q=n, strategy=E.GLOBAL, chi_max=a.chi_cap, fixed_chi=a.fixed_chi,
              precision=prec, log_truncations=False, stream=stream.cuda_stream, svd_kernel=svd_kernel_of(a, E),
              qr=qr_of(a, E))
    flush = torch.empty(a.flush_mb * (1 << 20) // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step_device():
        m.reset()
        E.mps_apply_circuit_device(m.h, qs, ops_dev.data_ptr(), 4)
        return m.fidelity()

    def step_host(pinned_ops):
        m.reset()
        for g in range(n):
            m.apply_2q(int(qs[g]), pinned_ops[g])
        return m.fidelity()

    for _ in range(a.warmup):
        step_device()
    # ---- timed region: inputs resident in HBM
    clocks = ClockSampler(local)
    m.stats_reset()
    m.profile(True)
    step_ms = []
    fid = None
    clocks.start()
    wall0 = time.perf_counter()
    for _ in range(a.steps):
        flush.fill_(1.0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fid = step_device()
        e1.record(stream)
        barrier()
        step_ms.append(e0.elapsed_time(e1))
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    m.profile(False)
    st = m.stats()
    bonds = m.bond_dims()
    total_s, total_updates = reduce_max_sum(sum(step_ms) / 1e3, float(n * a.steps), world, dev)
    value = total_updates / total_s
    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    e2e = None
    if not a.no_e2e:
        pinned = [np.ascontiguousarray(u) for u in circ.ops]
        e2e_ms = []
        for _ in range(a.steps):
            flush.fill_(1.0)
            barrier()
            t0 = time.perf_counter()
            step_host(pinned)
            barrier()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e_s, e_n = reduce_max_sum(sum(e2e_ms) / 1e3, float(n * a.steps), world, dev)
        e2e = {"value": e_n / e_s, "unit": "updates/s", "h2d_bytes_per_step": int(n * 16 * 16),
               "d2h_bytes_per_step": int(n * 160 + 8), "ms_per_step": statistics.mean(e2e_ms)}
    # ---- roofline of the dominant kernel (the Jacobi SVD, FP32 ALU bound)
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peak = fp32_peak_tflops(sm_count, 2070.0) if a.precision != "fp64" else None
    jac_s = st["jacobi_ms"] / 1e3
    achieved = (st["jacobi_flops"] / jac_s / 1e12) if jac_s > 0 else None
    # DRAM bytes of one 512 x 512 launch of the point-to-point kernel: dram__bytes_read.sum +
    # dram__bytes_write.sum of the ncu capture summarised in TRAFFIC_SOURCE (not measured by this
    # run); the algorithmic bytes of that launch are one read and one write of theta,
    # 2 x 512 x 512 x 8 B
    peaks = measured_peaks()
    tf32_peak = peaks.get("bf16_tflops", 1900.0) / 2.0   # the tf32 rate is half the bf16 rate
    roof = {"bound": "alu", "kernel": "jacobi_kernel3 and the other one-sided Jacobi SVD kernels, FP32",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if (achieved and peak) else None,
            "traffic": TRAFFIC_512 if a.precision != "fp64" else None,
            "traffic_launch": "jacobi_kernel3, theta 512 x 512 (bytes per launch; algorithmic 4194304)",
            "traffic_source": TRAFFIC_SOURCE,
            "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flops x 2070 MHz (derived, not measured)",
            "share_of_step": (st["jacobi_ms"] / sum(step_ms)) if step_ms else None,
            "launches": st["jacobi_launches"], "avg_launch_ms": st["jacobi_ms"] / max(st["jacobi_launches"], 1),
            "sweeps_per_launch": st["jacobi_sweeps"] / max(st["jacobi_launches"], 1),
            "centre_move_share": (st["move_jacobi_ms"] / st["jacobi_ms"]) if st["jacobi_ms"] else None}
    qr = {"launches": st["qr_launches"], "ms": st["qr_ms"],
          "share_of_step": (st["qr_ms"] / sum(step_ms)) if step_ms else None}
    gemm_tf = (st["gemm_flops"] / (st["gemm_ms"] / 1e3) / 1e12) if st["gemm_ms"] > 0 else None
    gemm = {"launches": st["gemm_launches"], "ms": st["gemm_ms"], "tflops": gemm_tf,
            "issued_tensor_tflops": 3 * gemm_tf if gemm_tf else None,
            "tensor_peak_tflops": tf32_peak,
            "tensor_peak_source": "tf32 = bf16 burst of the measured peaks / 2 (nominal ratio)"
                                  if "bf16_tflops" in peaks else "tf32 = fallback 1.9 PFLOP/s bf16 / 2"}
    # the contraction's share of the tensor pipe: 3xTF32 issues three products per useful one
    roof["contraction_frac"] = (3 * gemm_tf / tf32_peak) if gemm_tf else None
    extras = {}
    if rank == 0 and world == 1 and not a.no_extras:
        extras["time_to_target"] = time_to_target(E, torch, dev, a, prec)
        extras["chi512"] = chi512_throughput(E, torch, dev, a, prec, circ, ops_dev, qs)
        extras["precision_vs_fp64"] = precision_vs_fp64(E, a, prec, circ)
        extras["batch"] = batch_block(E, torch, dev, a, prec)
        extras["vidal_layers"] = vidal_layers_block(E, torch, dev, a, prec, circ, ops_dev, qs)
    extras["svd_layout_tuning"] = svd_tuning_summary(E)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_oracle_sample(circ, a, a.cpu_sample_s)
    if rank == 0:
        line = {"metric": "2-qubit MPS updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.mean(step_ms),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if a.precision == "fp64" else "f32",
                "data": "synthetic", "precision": a.precision,
                "config": bench_config(a, n, world),
                "inferred_fidelity": fid, "final_max_bond": max(bonds),
                "wall_s_timed": wall, "gpu_launches": st["kernel_launches"], "roofline": roof,
                "contraction": gemm, "householder_qr": qr, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "options": {"svd_kernel": a.svd_kernel, "qr": a.qr}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    m.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _timed_circuit(E, torch, dev, n_qubits, qs, ops_dev, op_dim, **mps_kw):
    """One run of a whole circuit from |0...0> (a pure state, or |0...0><0...0| for kind MIXED);
    returns (GPU ms, inferred fidelity, max bond, Jacobi ms, Jacobi launches)."""
    stream = torch.cuda.current_stream(dev)
    m = E.MPS(n_qubits, log_truncations=False, stream=stream.cuda_stream, **mps_kw)
    m.profile(True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    E.mps_apply_circuit_device(m.h, qs, ops_dev.data_ptr(), op_dim)
    fid = m.fidelity()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st = m.stats()
    out = (e0.elapsed_time(e1), fid, max(m.bond_dims()), st["jacobi_ms"], st["jacobi_launches"])
    m.close()
    return out


def time_to_target(E, torch, dev, a, prec) -> dict:
    """The paper's time-to-fidelity comparison ("Benchmarks"): an EA run at F_min on a circuit where
    the fidelity budget binds (the same 100-qubit chain, brickwork depth 8, same seed), then a
    fixed-bond run at the largest bond the EA run used.  Median GPU time of three runs each."""
    circ = W.brickwork_circuit(a.n_qubits, 8, a.seed)
    n = circ.n_2q
    ops_dev = torch.from_numpy(circ.ops_array().view(np.float64).reshape(n, 32).copy()).to(dev)
    qs = np.asarray(circ.qs, dtype=np.int32)
    kw = dict(precision=prec, svd_kernel=svd_kernel_of(a, E), qr=qr_of(a, E))
    ea = [_timed_circuit(E, torch, dev, a.n_qubits, qs, ops_dev, 4, f_min=a.f_min, n_2q=n, strategy=E.GLOBAL,
                         chi_max=a.chi_cap, **kw) for _ in range(3)]
    chi = ea[0][2]
    fx = [_timed_circuit(E, torch, dev, a.n_qubits, qs, ops_dev, 4, n_2q=n, fixed_chi=chi, chi_max=chi, **kw)
          for _ in range(3)]
    ea_s = statistics.median(r[0] for r in ea) / 1e3
    fx_s = statistics.median(r[0] for r in fx) / 1e3
    return {"workload": f"{a.n_qubits}-qubit chain, brickwork depth 8, Haar SU(4), seed {a.seed}, {n} gates",
            "f_min": a.f_min,
            "ea": {"gpu_s": ea_s, "inferred_fidelity": ea[0][1], "max_bond": chi,
                   "reached_f_min": bool(ea[0][1] >= a.f_min)},
            "fixed_chi": {"chi": chi, "gpu_s": fx_s, "inferred_fidelity": fx[0][1]},
            "ea_time_over_fixed": ea_s / fx_s}


def batch_block(E, torch, dev, a, prec, n_circuits: int = 16) -> dict:
    """Many independent circuits through mps_batch_run: the first n_circuits of the batch study's
    seeded mix (N ~ U[20, 80], depth ~ U[10, 30], F_min in {0.9, 0.99}, bond cap 128), one at a time
    and eight at a time; wall time, host threads included.  Each circuit's result must be the same
    at both concurrencies."""
    specs = W.random_batch_specs(64, a.seed)[:n_circuits]
    circs = [W.brickwork_circuit(sp["n_qubits"], sp["depth"], sp["seed"]) for sp in specs]
    devs = [torch.from_numpy(c.ops_array().view(np.float64).reshape(c.n_2q, 32).copy()).to(dev) for c in circs]
    total = sum(c.n_2q for c in circs)
    items = [{"n_qubits": sp["n_qubits"], "qs": c.qs, "ops_dev": dv.data_ptr(), "op_dim": 4, "f_min": sp["f_min"],
              "n_2q": c.n_2q, "chi_max": 128, "precision": prec} for sp, c, dv in zip(specs, circs, devs)]
    E.mps_batch_run(items[:2], concurrency=2)   # warm-up
    out = {"workload": f"{n_circuits} brickwork circuits, N ~ U[20, 80], depth ~ U[10, 30], F_min 0.9 / 0.99, "
                       f"bond cap 128 ({total} gates)", "gates": total}
    fids = {}
    for conc in (1, 8):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        code, res = E.mps_batch_run(items, concurrency=conc)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        fids[conc] = [r["fidelity"] for r in res]
        out[f"concurrency_{conc}"] = {"wall_s": dt, "updates_per_s": total / dt, "status": code}
    out["speedup"] = out["concurrency_1"]["wall_s"] / out["concurrency_8"]["wall_s"]
    out["same_results"] = fids[1] == fids[8]
    return out


def vidal_layers_block(E, torch, dev, a, prec, circ, ops_dev, qs, conc: int = 8) -> dict:
    """The benchmark circuit in Vidal form, the gates of each brickwork layer concurrently
    (mps_apply_layer_device, one schedule target per layer); wall time, host threads included."""
    n = circ.n_2q
    bounds = [0] + [g for g in range(1, n) if circ.layers[g] != circ.layers[g - 1]] + [n]
    m = E.MPS(a.n_qubits, f_min=a.f_min, n_2q=n, strategy=E.GLOBAL, chi_max=a.chi_cap, precision=prec,
              log_truncations=False, vidal=True)
    m.apply_layer(qs[:1], ops_dev.data_ptr(), concurrency=conc)   # warm-up: helper handles
    m.close()
    m = E.MPS(a.n_qubits, f_min=a.f_min, n_2q=n, strategy=E.GLOBAL, chi_max=a.chi_cap, precision=prec,
              log_truncations=False, vidal=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for a0, a1 in zip(bounds[:-1], bounds[1:]):
        m.apply_layer(qs[a0:a1], ops_dev.data_ptr() + a0 * 256, concurrency=conc)
    fid = m.fidelity()
    dt = time.perf_counter() - t0
    out = {"workload": f"same circuit, Vidal form, {len(bounds) - 1} layers, {conc} gates at a time",
           "concurrency": conc, "wall_s": dt, "updates_per_s": n / dt, "inferred_fidelity": fid,
           "max_bond": max(m.bond_dims()),
           "note": "Vidal form: no canonical centre, so the inferred product is not a fidelity estimate here"}
    m.close()
    return out


def svd_tuning_summary(E) -> dict:
    """The Jacobi layout autotuner's choices so far in this process (shape classes of the SVD,
    rows and columns rounded up to 64): how many classes were timed and where each layout won."""
    tab = E.mps_svd_tuning()

    def names(layout):
        return [f"{t['rows']}x{t['cols']}{'+W' if t['accumulate'] else ''}" for t in tab if t["layout"] == layout]

    ratios = [t["ms_gram"] / t["ms_tournament"] for t in tab if t["ms_gram"] > 0 and t["ms_tournament"] > 0]
    split = [t["ms_tournament"] / t["ms_unsplit"] for t in tab if t["ms_unsplit"] > 0 and t["ms_tournament"] > 0]
    return {"classes": len(tab), "gram_classes": names("gram"), "unsplit_classes": names("tournament_unsplit"),
            "gram_over_tournament_time": {"min": min(ratios), "max": max(ratios)} if ratios else None,
            "split_over_unsplit_time": {"min": min(split), "max": max(split)} if split else None}


def chi512_throughput(E, torch, dev, a, prec, circ, ops_dev, qs) -> dict:
    """Fixed bond 512 (the largest fixed-chi point of the pure-state benchmark) on the same circuit:
    every saturated update is a 1024 x 1024 SVD."""
    n = circ.n_2q
    # the saturated 1024 x 1024 SVD's layout is tuned before the clock starts (once per process)
    t = E.MPS(a.n_qubits, fixed_chi=512, chi_max=512, precision=prec, svd_kernel=svd_kernel_of(a, E), qr=qr_of(a, E))
    for acc in (False, True):
        t.svd_tune(1024, 1024, acc)
    t.close()
    ms, fid, mx, jms, jl = _timed_circuit(E, torch, dev, a.n_qubits, qs, ops_dev, 4, n_2q=n, fixed_chi=512,
                                          chi_max=512, precision=prec, svd_kernel=svd_kernel_of(a, E), qr=qr_of(a, E))
    return {"workload": f"same circuit, fixed chi = 512 ({n} gates)", "updates_per_s": n / (ms / 1e3),
            "gpu_s": ms / 1e3, "inferred_fidelity": fid, "max_bond": mx, "jacobi_share": jms / ms,
            "jacobi_ms_per_launch": jms / max(jl, 1)}


def precision_vs_fp64(E, a, prec, circ, n_prefix: int = 350) -> dict:
    """The complex64 path against the complex128 path on the GPU (MPS_FP64), on the first n_prefix
    gates of the benchmark circuit with the benchmark's schedule: the largest relative error of
    the retained singular values per gate, of the running product, and the overlap of the states."""
    n_prefix = min(n_prefix, circ.n_2q)
    runs = {}
    for name, pr in (("fp64", E.FP64), ("ours", prec)):
        m = E.MPS(a.n_qubits, f_min=a.f_min, n_2q=circ.n_2q, strategy=E.GLOBAL, chi_max=a.chi_cap, precision=pr,
                  svd_kernel=svd_kernel_of(a, E), qr=qr_of(a, E))
        sv = []
        for g in range(n_prefix):
            q, u = circ.gates()[g]
            m.apply_2q(q, u)
            sv.append(m.last_singular_values())
        runs[name] = (m, m.truncation_log(), sv)
    (m64, log64, sv64), (m32, log32, sv32) = runs["fp64"], runs["ours"]
    compared, rel = 0, 0.0
    for g64, g32, s64, s32 in zip(log64, log32, sv64, sv32):
        if g64["k"] != g32["k"]:
            break
        k = g64["k"]
        rel = max(rel, float(np.max(np.abs(s32[:k] - s64[:k]) / s64[:k])))
        compared += 1
    out = {"gates": n_prefix, "gates_with_equal_bonds": compared, "max_bond": max(m64.bond_dims()),
           "max_rel_err_retained_s": rel, "product_fp64": m64.fidelity(), "product_ours": m32.fidelity(),
           "abs_err_product": abs(m64.fidelity() - m32.fidelity()),
           "overlap_with_fp64": abs(m64.overlap(m32)) ** 2}
    m64.close()
    m32.close()
    return out


def run_study(a) -> int:
    """Measurement studies on one GPU, one JSON line per run and a summary line.

    ttf: the paper's time-to-fidelity methodology (EA run at F_min records its
    largest bond; fixed-bond runs at that bond and at 128/256/512), on 100-qubit
    Haar brickworks of depth 8 (EA reaches F_min below the cap) and depth 30
    (every run is cap-bound).  mpo: the noisy 30-qubit depth-15 brickwork as a
    density matrix (d = 4): every gate fused with two-qubit depolarising noise
    p = 0.01 and amplitude damping gamma = 0.005 on both qubits, F_min = 0.95.
    batch: 64 independent brickworks (N ~ U[20, 80], depth ~ U[10, 30], F_min in
    {0.9, 0.99}, bond cap 128) through mps_batch_run at concurrency 1, 4, 8, 16;
    wall time of the whole batch (host threads included).  strategies: an 18-qubit
    depth-18 brickwork at F_min 0.9 and 0.5 under each schedule; the true
    fidelity |<exact|EA>|^2 comes from mps_overlap with the untruncated run.  grad: the
    parameter-shift gradient (2P + 1 circuits) of sum_i <Z_i Z_{i+1}> for the layered ansatz,
    20 qubits x 3 layers untruncated and 40 qubits x 2 layers at F_min 0.99, as one batch.
    vidal: inferred against true fidelity of the canonical and the Vidal/Hastings form (18 qubits,
    depth 18), their throughput on the 100-qubit depth-30 circuit, and the Vidal form run layer
    by layer with the gates of a layer concurrent (concurrency 1, 4, 8, 16; wall time).
    """
    import torch
    import paper_2307_16870_gb300 as E
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prec = {"tf32x3": E.TF32X3, "fp32": E.FP32, "fp64": E.FP64}[a.precision]
    rows = []

    def emit(row):
        rows.append(row)
        print(json.dumps(row), flush=True)

    if a.study == "ttf":
        for depth in (8, 30):
            circ = W.brickwork_circuit(100, depth, a.seed)
            n = circ.n_2q
            ops_dev = torch.from_numpy(circ.ops_array().view(np.float64).reshape(n, 32).copy()).to(dev)
            qs = np.asarray(circ.qs, dtype=np.int32)
            # warm-up (kernel loading, allocation)
            _timed_circuit(E, torch, dev, 100, qs[:50], ops_dev, 4, f_min=0.9, n_2q=n, chi_max=64, precision=prec)
            for f_min in (0.9, 0.5):
                for cap in (256, 512):
                    ms, fid, mx, jms, jl = _timed_circuit(E, torch, dev, 100, qs, ops_dev, 4, f_min=f_min, n_2q=n,
                                                          strategy=E.GLOBAL, chi_max=cap, precision=prec)
                    emit({"study": "ttf", "depth": depth, "n_2q": n, "mode": "EA", "f_min": f_min, "chi_cap": cap,
                          "gpu_s": ms / 1e3, "updates_per_s": n / (ms / 1e3), "inferred_fidelity": fid,
                          "max_bond": mx, "reached_f_min": bool(fid >= f_min), "jacobi_share": jms / ms})
            chis = sorted({128, 256, 512} | {r["max_bond"] for r in rows if r.get("depth") == depth})
            for chi in chis:
                ms, fid, mx, jms, jl = _timed_circuit(E, torch, dev, 100, qs, ops_dev, 4, n_2q=n, fixed_chi=chi,
                                                      chi_max=chi, precision=prec)
                emit({"study": "ttf", "depth": depth, "n_2q": n, "mode": "fixed", "chi": chi, "gpu_s": ms / 1e3,
                      "updates_per_s": n / (ms / 1e3), "inferred_fidelity": fid, "max_bond": mx,
                      "jacobi_share": jms / ms})
    elif a.study == "mpo":
        n_q, depth, p, gamma = 30, 15, 0.01, 0.005
        circ = W.brickwork_circuit(n_q, depth, a.seed)
        n = circ.n_2q
        ad = E.mps_superop_from_kraus(W.amplitude_damping_kraus(gamma), 1)
        dep = E.mps_superop_from_kraus(W.depolarizing_2q_kraus(p), 2)
        ops = np.stack([np.kron(ad, ad) @ dep @ E.mps_superop_from_kraus([u], 2) for u in circ.ops])
        ops_dev = torch.from_numpy(np.ascontiguousarray(ops).view(np.float64).reshape(n, 512).copy()).to(dev)
        qs = np.asarray(circ.qs, dtype=np.int32)
        _timed_circuit(E, torch, dev, n_q, qs[:20], ops_dev, 16, kind=E.MIXED, f_min=0.95, n_2q=n, chi_max=64,
                       precision=prec)
        for mixed_fid in (E.KEPT_RATIO, E.WANG_SQRT):
            for cap in (128, 256):
                ms, fid, mx, jms, jl = _timed_circuit(E, torch, dev, n_q, qs, ops_dev, 16, kind=E.MIXED, f_min=0.95,
                                                      n_2q=n, strategy=E.GLOBAL, chi_max=cap, precision=prec,
                                                      mixed_fid=mixed_fid)
                emit({"study": "mpo", "n_qubits": n_q, "depth": depth, "n_2q": n, "p_depol": p, "gamma_ad": gamma,
                      "f_min": 0.95, "mixed_fid": "kept_ratio" if mixed_fid == E.KEPT_RATIO else "wang_sqrt",
                      "chi_cap": cap, "gpu_s": ms / 1e3, "updates_per_s": n / (ms / 1e3),
                      "inferred_fidelity": fid, "max_bond": mx, "jacobi_share": jms / ms})
    elif a.study == "strategies":
        n_q, depth = 18, 18
        circ = W.brickwork_circuit(n_q, depth, a.seed)
        n = circ.n_2q
        ops_dev = torch.from_numpy(circ.ops_array().view(np.float64).reshape(n, 32).copy()).to(dev)
        qs = np.asarray(circ.qs, dtype=np.int32)
        exact = E.MPS(n_q, n_2q=n, precision=prec, log_truncations=False)
        E.mps_apply_circuit_device(exact.h, qs, ops_dev.data_ptr(), 4, 1.0)     # untruncated reference
        names = {E.NAIVE: "naive", E.GLOBAL: "global", E.NEAREST: "nearest"}
        for f_min in (0.9, 0.5):
            for strat in (E.NAIVE, E.GLOBAL, E.NEAREST):
                stream = torch.cuda.current_stream(dev)
                m = E.MPS(n_q, f_min=f_min, n_2q=n, strategy=strat, precision=prec, log_truncations=False,
                          stream=stream.cuda_stream)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                E.mps_apply_circuit_device(m.h, qs, ops_dev.data_ptr(), 4)
                inferred = m.fidelity()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                true_f = abs(exact.overlap(m)) ** 2
                emit({"study": "strategies", "n_qubits": n_q, "depth": depth, "n_2q": n, "f_min": f_min,
                      "strategy": names[strat], "inferred_fidelity": inferred, "true_fidelity": true_f,
                      "gpu_s": e0.elapsed_time(e1) / 1e3, "max_bond": max(m.bond_dims()),
                      "exact_max_bond": max(exact.bond_dims())})
                m.close()
        exact.close()
    elif a.study == "e1":
        # Fig. 1 rerun at 25 qubits, depth 20: naive / global / nearest schedules at F_min 0.9 and
        # 0.5, and the bond-cap trade-off (global, F_min 0.9, caps 64..512).  The true fidelity
        # |<exact|EA>|^2 takes the exact state from a dense state-vector evolution (2^25 complex128
        # amplitudes, 512 MB on the GPU, PyTorch tensor operations: measurement only, not the
        # library's path) and contracts it with the EA state's sites.
        n_q, depth = 25, 20
        circ = W.brickwork_circuit(n_q, depth, a.seed)
        n = circ.n_2q
        ops_dev = torch.from_numpy(circ.ops_array().view(np.float64).reshape(n, 32).copy()).to(dev)
        qs = np.asarray(circ.qs, dtype=np.int32)
        psi = torch.zeros(2 ** n_q, dtype=torch.complex128, device=dev)
        psi[0] = 1.0
        for q, u in circ.gates():
            ut = torch.from_numpy(np.ascontiguousarray(u)).to(dev)
            v = psi.view(2 ** q, 4, 2 ** (n_q - q - 2))
            psi = torch.einsum("ab,ibj->iaj", ut, v).reshape(-1)
        torch.cuda.synchronize(dev)

        def true_fidelity(m):
            # <exact|m>: contract conj(psi) site by site, left to right
            t = psi.conj().view(1, 2, -1)                     # (chi=1, sigma, rest)
            for i in range(n_q):
                site = torch.from_numpy(m.site(i)).to(dev)     # (chi_l, 2, chi_r)
                t = torch.einsum("lsr,lsk->rk", site, t)       # (chi_r, rest)
                if i + 1 < n_q:
                    t = t.reshape(t.shape[0], 2, -1)
            return float(abs(t.reshape(-1)[0]) ** 2)

        names = {E.NAIVE: "naive", E.GLOBAL: "global", E.NEAREST: "nearest"}
        runs = [("strategy", f_min, strat, 512) for f_min in (0.9, 0.5) for strat in (E.NAIVE, E.GLOBAL, E.NEAREST)]
        runs += [("chi_cap", 0.9, E.GLOBAL, cap) for cap in (64, 128, 256, 512)]
        _timed_circuit(E, torch, dev, n_q, qs[:30], ops_dev, 4, f_min=0.9, n_2q=n, chi_max=64, precision=prec)
        for kind, f_min, strat, cap in runs:
            stream = torch.cuda.current_stream(dev)
            m = E.MPS(n_q, f_min=f_min, n_2q=n, strategy=strat, chi_max=cap, precision=prec, log_truncations=True,
                      stream=stream.cuda_stream)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E.mps_apply_circuit_device(m.h, qs, ops_dev.data_ptr(), 4)
            inferred = m.fidelity()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            log = m.truncation_log()
            emit({"study": "e1", "part": kind, "n_qubits": n_q, "depth": depth, "n_2q": n, "f_min": f_min,
                  "strategy": names[strat], "chi_cap": cap, "inferred_fidelity": inferred,
                  "true_fidelity": true_fidelity(m), "gpu_s": e0.elapsed_time(e1) / 1e3,
                  "max_bond": max(m.bond_dims()), "cap_hits": sum(1 for r in log if r["cap_hit"])})
            m.close()
    elif a.study == "vidal":
        # (1) inferred against true fidelity, canonical and Vidal form, 18 qubits depth 18
        n_q, depth = 18, 18
        circ = W.brickwork_circuit(n_q, depth, a.seed)
        n = circ.n_2q
        ops_dev = torch.from_numpy(circ.ops_array().view(np.float64).reshape(n, 32).copy()).to(dev)
        qs = np.asarray(circ.qs, dtype=np.int32)
        exact = E.MPS(n_q, n_2q=n, precision=prec, log_truncations=False)
        E.mps_apply_circuit_device(exact.h, qs, ops_dev.data_ptr(), 4, 1.0)
        for f_min in (0.9, 0.5):
            for vid in (False, True):
                m = E.MPS(n_q, f_min=f_min, n_2q=n, precision=prec, log_truncations=False, vidal=vid)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                E.mps_apply_circuit_device(m.h, qs, ops_dev.data_ptr(), 4)
                inferred = m.fidelity()
                dt = time.perf_counter() - t0
                ov = exact.overlap(m)
                nrm = m.overlap(m).real
                emit({"study": "vidal", "n_qubits": n_q, "depth": depth, "f_min": f_min,
                      "form": "vidal" if vid else "canonical", "inferred_fidelity": inferred,
                      "true_fidelity": abs(ov) ** 2 / nrm, "norm2": nrm, "wall_s": dt,
                      "max_bond": max(m.bond_dims())})
                m.close()
        exact.close()
        # (2) throughput on the 100-qubit depth-30 circuit, cap 256
        circ = W.brickwork_circuit(100, 30, a.seed)
        n = circ.n_2q
        ops_dev = torch.from_numpy(circ.ops_array().view(np.float64).reshape(n, 32).copy()).to(dev)
        qs = np.asarray(circ.qs, dtype=np.int32)
        for vid in (False, True):
            ms, fid, mx, jms, jl = _timed_circuit(E, torch, dev, 100, qs, ops_dev, 4, f_min=0.9, n_2q=n,
                                                  strategy=E.GLOBAL, chi_max=256, precision=prec, vidal=vid)
            emit({"study": "vidal", "n_qubits": 100, "depth": 30, "f_min": 0.9, "chi_cap": 256,
                  "form": "vidal" if vid else "canonical", "gpu_s": ms / 1e3, "updates_per_s": n / (ms / 1e3),
                  "inferred_fidelity": fid, "max_bond": mx, "jacobi_share": jms / ms})
        # (3) the Vidal form layer by layer, the gates of each layer concurrently (one target per
        # layer); wall time including the host threads
        bounds = [0] + [g for g in range(1, n) if circ.layers[g] != circ.layers[g - 1]] + [n]
        for conc in (1, 4, 8, 16):
            m = E.MPS(100, f_min=0.9, n_2q=n, strategy=E.GLOBAL, chi_max=256, precision=prec,
                      log_truncations=False, vidal=True)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for a0, a1 in zip(bounds[:-1], bounds[1:]):
                m.apply_layer(qs[a0:a1], ops_dev.data_ptr() + a0 * 256, concurrency=conc)
            fid = m.fidelity()
            dt = time.perf_counter() - t0
            emit({"study": "vidal", "n_qubits": 100, "depth": 30, "f_min": 0.9, "chi_cap": 256,
                  "form": "vidal_layers", "concurrency": conc, "wall_s": dt, "updates_per_s": n / dt,
                  "inferred_fidelity": fid, "max_bond": max(m.bond_dims())})
            m.close()
    elif a.study == "precision":
        # the same circuits in complex128 (FP64 throughout) and in the two complex64 modes: the
        # error of each result against the FP64-on-GPU run
        def _run(n_q, circ, op_dim, ops_dev, kind, f_min, cap, pr):
            qs = np.asarray(circ.qs, dtype=np.int32)
            m = E.MPS(n_q, kind=kind, f_min=f_min, n_2q=circ.n_2q, chi_max=cap, precision=pr)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            E.mps_apply_circuit_device(m.h, qs, ops_dev.data_ptr(), op_dim)
            fid = m.fidelity()
            return m, time.perf_counter() - t0, fid
        names = {E.FP64: "fp64", E.FP32: "fp32", E.TF32X3: "tf32x3"}
        pure = W.brickwork_circuit(30, 16, a.seed)
        pure_ops = torch.from_numpy(pure.ops_array().view(np.float64).reshape(pure.n_2q, 32).copy()).to(dev)
        mpo = W.brickwork_circuit(12, 8, a.seed)
        ad = E.mps_superop_from_kraus(W.amplitude_damping_kraus(0.005), 1)
        dep = E.mps_superop_from_kraus(W.depolarizing_2q_kraus(0.01), 2)
        sops = np.stack([np.kron(ad, ad) @ dep @ E.mps_superop_from_kraus([u], 2) for u in mpo.ops])
        mpo_ops = torch.from_numpy(np.ascontiguousarray(sops).view(np.float64).reshape(mpo.n_2q, 512).copy()).to(dev)
        for label, n_q, circ, op_dim, ops_dev, kind, f_min, cap in (
                ("pure 30q D16", 30, pure, 4, pure_ops, E.PURE, 0.99, 64),
                ("mpo 12q D8 noisy", 12, mpo, 16, mpo_ops, E.MIXED, 0.95, 64)):
            ref, t_ref, f_ref = _run(n_q, circ, op_dim, ops_dev, kind, f_min, cap, E.FP64)
            b_ref = ref.bond_dims()
            nrm = ref.overlap(ref).real
            for pr in (E.FP64, E.FP32, E.TF32X3):
                m, dt, fid = (ref, t_ref, f_ref) if pr == E.FP64 else _run(n_q, circ, op_dim, ops_dev, kind, f_min,
                                                                           cap, pr)
                ov = ref.overlap(m)
                bd = m.bond_dims()
                emit({"study": "precision", "circuit": label, "precision": names[pr], "f_min": f_min, "chi_cap": cap,
                      "wall_s": dt, "updates_per_s": circ.n_2q / dt, "inferred_fidelity": fid,
                      "abs_fidelity_diff_vs_fp64": abs(fid - f_ref),
                      "overlap_vs_fp64": float(abs(ov) ** 2 / (nrm * m.overlap(m).real)),
                      "bonds_equal_fp64": int(sum(x == y for x, y in zip(bd, b_ref))), "bonds": len(bd)})
                if m is not ref:
                    m.close()
            ref.close()
        # the differentiable form: complex64 reverse mode against the FP64 one
        from paper_2307_16870_gb300 import autodiff as AD
        for n_q, layers, f_min in ((20, 3, 1.0), (20, 3, 0.95)):
            p = W.ansatz_params(n_q, layers, a.seed)
            e64, g64, _ = AD.energy_and_grad_ad(n_q, layers, p, f_min=f_min, chi_max=64, precision=E.FP64)
            for pr in (E.TF32X3, E.FP32):
                e, g, info = AD.energy_and_grad_ad(n_q, layers, p, f_min=f_min, chi_max=64, precision=pr)
                emit({"study": "precision", "circuit": "reverse mode, ansatz %dq x %d layers" % (n_q, layers),
                      "precision": names[pr], "f_min": f_min, "energy_diff_vs_fp64": abs(e - e64),
                      "grad_max_abs_diff_vs_fp64": float(np.abs(g - g64).max()),
                      "grad_norm": float(np.linalg.norm(g64))})
    elif a.study == "grad":
        from paper_2307_16870_gb300 import grad as G
        for n_q, layers, f_min, cap in ((20, 3, 1.0, 0), (40, 2, 0.99, 64)):
            p = W.ansatz_params(n_q, layers, a.seed)
            fn = (lambda nq, ly: (lambda ang: W.ansatz_circuit(nq, ly, ang)))(n_q, layers)
            G.energy_and_grad(fn, n_q, p, f_min=f_min, chi_max=cap, concurrency=8, with_grad=False)   # warm-up
            for conc in (1, 8):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                e, g, info = G.energy_and_grad(fn, n_q, p, f_min=f_min, chi_max=cap, concurrency=conc)
                torch.cuda.synchronize(dev)
                dt = time.perf_counter() - t0
                emit({"study": "grad", "n_qubits": n_q, "layers": layers, "params": int(p.size), "f_min": f_min,
                      "chi_cap": cap, "concurrency": conc, "circuits": info["circuits"], "updates": info["updates"],
                      "wall_s": dt, "updates_per_s": info["updates"] / dt, "energy": e,
                      "grad_norm": float(np.linalg.norm(g)),
                      "min_inferred_fidelity": float(min(info["inferred_fidelity"]))})
            g_ps = g
            # reverse mode through the same truncated simulation (one forward, one backward)
            from paper_2307_16870_gb300 import autodiff as AD
            AD.energy_and_grad_ad(n_q, layers, p, f_min=f_min, chi_max=cap or 256)       # warm-up
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            e, g, info = AD.energy_and_grad_ad(n_q, layers, p, f_min=f_min, chi_max=cap or 256)
            dt = time.perf_counter() - t0
            emit({"study": "grad", "method": "reverse_mode", "n_qubits": n_q, "layers": layers,
                  "params": int(p.size), "f_min": f_min, "chi_cap": cap, "wall_s": dt,
                  "forward_s": info["forward_s"], "backward_s": info["backward_s"],
                  "svd_updates": info["updates"], "energy": e, "grad_norm": float(np.linalg.norm(g)),
                  "max_abs_diff_vs_parameter_shift": float(np.abs(g - g_ps).max()),
                  "inferred_fidelity": info["fidelity"], "max_bond": info["max_bond"]})
        # the 40-qubit, 10-layer ansatz at F_min 0.99 by reverse mode only (parameter shift would
        # take 2 * 1190 + 1 circuits)
        from paper_2307_16870_gb300 import autodiff as AD
        n_q, layers, f_min, cap = 40, 10, 0.99, 64
        p = W.ansatz_params(n_q, layers, a.seed)
        for ckpt in (False, True):
            torch.cuda.synchronize(dev)
            torch.cuda.reset_peak_memory_stats(dev)
            base = torch.cuda.memory_allocated(dev)
            t0 = time.perf_counter()
            e, g, info = AD.energy_and_grad_ad(n_q, layers, p, f_min=f_min, chi_max=cap, checkpoint=ckpt)
            dt = time.perf_counter() - t0
            emit({"study": "grad", "method": "reverse_mode", "checkpoint_per_layer": ckpt, "n_qubits": n_q,
                  "layers": layers, "params": int(p.size), "f_min": f_min, "chi_cap": cap, "wall_s": dt,
                  "forward_s": info["forward_s"], "backward_s": info["backward_s"], "svd_updates": info["updates"],
                  "svd_calls_with_recompute": info["tsvd_calls"], "energy": e,
                  "grad_norm": float(np.linalg.norm(g)), "inferred_fidelity": info["fidelity"],
                  "max_bond": info["max_bond"],
                  "peak_tensor_bytes": int(torch.cuda.max_memory_allocated(dev) - base)})
    elif a.study == "batch":
        specs = W.random_batch_specs(64, a.seed)
        cap = 128
        circs, devs = [], []
        for sp in specs:
            c = W.brickwork_circuit(sp["n_qubits"], sp["depth"], sp["seed"])
            circs.append(c)
            devs.append(torch.from_numpy(c.ops_array().view(np.float64).reshape(c.n_2q, 32).copy()).to(dev))
        total = sum(c.n_2q for c in circs)
        items = [{"n_qubits": sp["n_qubits"], "qs": c.qs, "ops_dev": dv.data_ptr(), "op_dim": 4,
                  "f_min": sp["f_min"], "n_2q": c.n_2q, "chi_max": cap, "precision": prec}
                 for sp, c, dv in zip(specs, circs, devs)]
        E.mps_batch_run(items[:4], concurrency=4)          # warm-up (kernel loading)
        base = None
        for conc in (1, 4, 8, 16):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            code, res = E.mps_batch_run(items, concurrency=conc)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            fids = [r["fidelity"] for r in res]
            if base is None:
                base = fids
            emit({"study": "batch", "circuits": len(items), "gates": total, "chi_cap": cap, "concurrency": conc,
                  "wall_s": dt, "updates_per_s": total / dt, "status": code,
                  "same_fidelities_as_sequential": fids == base,
                  "reached_f_min": sum(1 for r, sp in zip(res, specs) if r["fidelity"] >= sp["f_min"]),
                  "max_bond": max(r["max_bond"] for r in res)})
    print(json.dumps({"study": a.study, "runs": len(rows), "precision": a.precision,
                      "device": torch.cuda.get_device_name(dev)}), flush=True)
    return 0


def qr_of(a, E) -> int:
    return {"moves": E.QR_MOVES, "precondition": E.QR_PRECONDITION, "both": E.QR_MOVES | E.QR_PRECONDITION,
            "none": 0}[a.qr]


def svd_kernel_of(a, E) -> int:
    return {"auto": E.SVD_AUTO, "tournament": E.SVD_TOURNAMENT, "tournament-unsplit": E.SVD_TOURNAMENT_UNSPLIT,
            "gram": E.SVD_GRAM}[a.svd_kernel]


def run_micro(a) -> int:
    """Per-launch Jacobi timing of saturated updates (used for focused profiling)."""
    import torch
    import paper_2307_16870_gb300 as E
    prec = {"tf32x3": E.TF32X3, "fp32": E.FP32, "fp64": E.FP64}[a.precision]
    chi, n = a.micro, 24
    q = n // 2 - (a.steps + 1 if a.micro_moves else 0)
    sites, _ = W.random_canonical_mps(n, chi, q, seed=7)
    m = E.MPS(n, chi_max=chi, fixed_chi=chi, precision=prec, log_truncations=False, svd_kernel=svd_kernel_of(a, E),
              qr=qr_of(a, E))
    m.load_sites(sites, q)
    m.profile(True)
    for g in range(max(a.steps, 1) + 1):
        pos = q + (2 * g if a.micro_moves else 0)
        m.apply_2q(min(pos, n - 2), W.haar_unitary(4, 3, g), 1.0)
    torch.cuda.synchronize()
    st = m.stats()
    jl = max(st["jacobi_launches"], 1)
    print(json.dumps({"micro_chi": chi, "svd_kernel": a.svd_kernel, "moves": bool(a.micro_moves),
                      "qr_launches": st["qr_launches"],
                      "jacobi_ms_per_launch": st["jacobi_ms"] / jl,
                      "qr_ms_per_launch": st["qr_ms"] / max(st["qr_launches"], 1),
                      "sweeps_per_launch": st["jacobi_sweeps"] / jl,
                      "jacobi_tflops": st["jacobi_flops"] / (st["jacobi_ms"] / 1e3) / 1e12 if st["jacobi_ms"] else None}))
    m.close()
    return 0


def main(argv=None) -> int:
    a = parse_args(argv)
    if a.micro:
        return run_micro(a)
    if a.study:
        return run_study(a)
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
