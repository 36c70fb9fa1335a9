"""Throughput of the VMC hot path on GB300: local energies per second.

One step is one pass of the whole hot path over one batch of walkers:
one Metropolis sweep (mcmc_step, Sec. 5), the local energies with value,
Jacobian and Laplacian propagation (local_energy, Eq. 31), the clipped
gradient weights (vmc_loss_weights, Sec. 4.4) and the weighted parameter
gradient of log|psi| (grad_logpsi, Eq. 30) when the library provides it.
``value`` = walkers processed per second over the timed steps (one local
energy per walker per step), inputs resident in HBM; ``e2e`` = the same
through the public API with host buffers and the copies inside the timed
region.  Walkers are independent Markov chains, so with several GPUs each
rank runs its own walkers (weak scaling, no collective on the data path).

``--impl reference`` times the FP64 CPU oracle instead (host cores, bounded
walker sample per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "local energies/sec (walker evals/s)"
UNIT = "local_energies/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="n2_fp32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay of the step")
    p.add_argument("--no-mala", action="store_true", help="skip the step with the Langevin sampler")
    p.add_argument("--no-batch", action="store_true", help="skip the uneven-molecule batch")
    p.add_argument("--no-natgrad", action="store_true", help="skip the natural-gradient direction")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default tile set (for runs under a profiler, which distorts the autotuner's timings)")
    p.add_argument("--no-pp", action="store_true", help="skip the pseudopotential and ansatz-variant legs")
    p.add_argument("--mala-tau", type=float, default=0.1, help="Langevin time step (bohr^2)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--profile-case", type=int, default=0, metavar="B",
                   help="run one call on B walkers of the workload and exit (small case for ncu)")
    p.add_argument("--profile-op", default="local_energy", choices=["local_energy", "grad", "mcmc"])
    p.add_argument("--profile-precision", default=None, choices=["fp64", "fp32", "bf16"],
                   help="precision of the profile case (default: the workload's)")
    p.add_argument("--msg-ib", type=int, default=0, choices=[0, 4, 8],
                   help="profile case: receivers per warp task of the jet message kernel (0: library default)")
    return p.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_config(wl, world):
    s, c = wl.system, wl.cfg
    return {"workload": f"{wl.system.name} {s.n_elec}e, D={c.width}, L={c.n_layers}, K={c.n_det}, "
                        f"{wl.B} walkers/GPU, {wl.precision.upper()}",
            "molecule": s.name, "electrons": s.n_elec, "width": c.width, "layers": c.n_layers,
            "det_pairs": c.n_det, "walkers_per_gpu": wl.B, "global_walkers": wl.B * world,
            "precision": wl.precision, "parallelism": f"walker-sharded x{world}"}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def oracle_sample(wl, seconds, threads=None):
    """Times the FP64 oracle's local energy on a bounded walker sample (inputs rounded to the
    workload's precision, so that the outputs are also the parity reference of those walkers).
    Returns (walkers, seconds, threads, theta, r, oracle outputs)."""
    import numpy as np

    import oracle
    from paper_2307_14123_gb300 import fixtures as fx

    oracle.build()
    cores = threads or os.cpu_count() or 1
    oracle.Oracle.set_threads(cores)
    o = oracle.Oracle(wl.system, wl.cfg)
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed)
    if wl.precision != "fp64":
        theta = theta.astype(np.float32).astype(np.float64)
    n = cores
    while True:
        r = fx.init_walkers(wl.system, n, wl.walker_seed)
        if wl.precision != "fp64":
            r = r.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        ref = o.local_energy(theta, r, with_grad=True)
        dt = time.perf_counter() - t0
        if dt * 2 > seconds or n >= wl.B:
            return n, dt, oracle.Oracle.threads(), theta, r, ref, o
        n = min(wl.B, n * max(2, int(seconds / max(dt, 1e-3) / 2)))


def oracle_leg(h, wl, seconds, dev, with_grad):
    """The oracle on the host cores: the CPU baseline (all cores, and one core on a smaller sample)
    and, from the same oracle outputs, the error of the GPU path on those walkers (log|psi|, E_loc,
    and the weighted gradient of log|psi| along random parameter directions)."""
    import numpy as np
    import torch

    import oracle

    n, dtc, cores, theta, r, ref, o = oracle_sample(wl, seconds)
    # one core, on a sample sized to ~a quarter of the budget
    n1 = max(1, min(n, int(n * seconds / 4 / max(dtc * cores, 1e-3))))
    oracle.Oracle.set_threads(1)
    t0 = time.perf_counter()
    o.local_energy(theta, r[:n1])
    dt1 = time.perf_counter() - t0
    oracle.Oracle.set_threads(cores)
    tdt = torch.float64 if wl.precision == "fp64" else torch.float32
    th_d = torch.tensor(theta, dtype=tdt, device=dev)
    r_d = torch.tensor(r, dtype=tdt, device=dev)
    la, sg, el = (x.cpu().numpy() for x in h.local_energy(th_d, r_d))
    la, el = la.astype(np.float64), el.astype(np.float64)
    S = 0.5 * (np.abs(ref["lap"]) + np.sum(ref["grad"] ** 2, axis=1))
    d_la, d_e = np.abs(la - ref["logabs"]), np.abs(el - ref["e_loc"])
    parity = {"walkers": int(n),
              "logabs": {"max_abs_err": float(d_la.max()), "mean_abs_err": float(d_la.mean()),
                         "max_rel_err": float(np.max(d_la / np.maximum(1, np.abs(ref["logabs"])))),
                         "frac_within_1e-5_rel": float(np.mean(d_la <= 1e-5 * np.maximum(1, np.abs(ref["logabs"]))))},
              "e_loc": {"max_abs_err": float(d_e.max()), "mean_abs_err": float(d_e.mean()),
                        "mean_err": float(np.mean(el - ref["e_loc"])), "max_err_over_S_b": float(np.max(d_e / S)),
                        "frac_within_contract": float(np.mean(d_e <= np.maximum(1e-4, 1e-5 * S))),
                        "frac_within_1e-4_Ha": float(np.mean(d_e <= 1e-4))},
              "sign_equal": float(np.mean(sg == ref["sign"])),
              "contract": "log|psi| 1e-5 max(1,|log|psi||), E_loc max(1e-4 Ha, 1e-5 S_b), S_b the size of the "
                          "kinetic terms; exceptions only at near-nodal walkers (tests/fp32_contract.py)"}
    if with_grad:
        k = min(n, 16)
        w = np.random.default_rng(0).normal(size=k) / k
        dirs = np.random.default_rng(1).normal(size=(2, o.P))
        G = h.grad_logpsi(th_d, r_d[:k].contiguous(), torch.tensor(w, dtype=tdt, device=dev), 0)
        g_dir = G.double().cpu().numpy() @ dirs.T
        jv = o.grad_jvp(theta, r[:k], dirs)
        ref_dir = w @ jv
        scale = np.abs(w) @ np.abs(jv)
        parity["grad_direction"] = {"walkers": k, "directions": 2,
                                    "max_rel_err": float(np.max(np.abs(g_dir - ref_dir) / scale)),
                                    "note": "sum_b w_b d log|psi_b| / d theta . v against the oracle's dual-number "
                                            "derivatives, relative to sum_b |w_b| |d log|psi_b| . v|"}
    cpu = {"value": n / dtc, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
           "single_thread": {"value": n1 / dt1, "unit": UNIT, "walkers": n1, "seconds": dt1},
           "sample": f"FP64 oracle local_energy on {n} of the {wl.B} walkers ({dtc:.1f} s on {cores} threads; "
                     f"{n1} walkers on one thread in {dt1:.1f} s); the oracle has no reverse mode, so its "
                     f"Metropolis and gradient legs are not included"}
    return cpu, parity


def run_reference(args):
    from paper_2307_14123_gb300 import fixtures as fx

    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    wl = fx.workload(args.workload)
    # size one step to ~4 s of host time so the whole run stays within minutes
    n, dt, cores = oracle_sample(wl, 8.0)[:3]
    per_walker = dt / n
    step_n = max(1, min(wl.B, int(round(4.0 / per_walker))))
    import numpy as np

    import oracle

    o = oracle.Oracle(wl.system, wl.cfg)
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed)
    r = fx.init_walkers(wl.system, step_n, wl.walker_seed)
    for _ in range(args.warmup):
        o.local_energy(theta, r)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.local_energy(theta, r)
    total = time.perf_counter() - t0
    value = step_n * args.steps / total
    sample = f"oracle local_energy on {step_n} of the {wl.B} walkers per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded walkers and random-init weights)",
            "config": workload_config(wl, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        import torch

        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        sel = []
        try:
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# dram__bytes_read.sum + dram__bytes_write.sum of the jet message kernel (layer >= 1 launch) per walker,
# from an ncu capture of the layer-1 launch on 512 N2 walkers (FP32, the tuned 4-receiver tile; summary under profiles/); None
# once the kernel has changed since that capture.
MSG_DRAM_BYTES_PER_WALKER = (263.570432e6 + 432.803840e6) / 512
# the same for one launch of the fused layer kernel (layer 1 of N2, 512 walkers, the receiver-pair
# producer design; summary under profiles/); None once the kernel has changed since that capture.
# Layer 0 (constant node channels) reads no z slabs and moves less.
LAYER_FUSED_DRAM_BYTES_PER_WALKER = (238.052864e6 + 108.800256e6) / 512
# the same for one launch of the sender-tiled message kernel (layer 1 of C4H4 in BF16 mode, 256
# walkers; summary under profiles/); None once the kernel has changed since that capture.
MSG_LARGE_DRAM_BYTES_PER_WALKER = (1.637387e9 + 0.949968e9) / 256


def gemm_shapes(wl, chunk):
    """(rows, K, n_out) of the forward GEMM kinds for one launch over `chunk` walkers (jets), and the
    value-only forward GEMM FLOPs per walker (the reverse pass repeats each product twice: the input
    adjoint and the weight gradient)."""
    s, c = wl.system, wl.cfg
    N, D, M, K = s.n_elec, c.width, s.n_nuc, c.n_det
    C = 3 * N + 2
    E = N * (N - 1) // 2 + N * M
    nsq = s.n_up ** 2 + s.n_down ** 2 if not c.full_det else 2 * N * N
    shapes = {"jet.gemm_update": (chunk * N * C, 3 * D, D), "jet.gemm_node": (chunk * N * C, D, D),
              "jet.gemm_edge": (chunk * E * 3, D, D),
              # per spin s: (n_s * C rows) x (K * n_s outputs), summed over both spins
              "jet.gemm_orbital": (chunk * C, D, K * nsq)}
    L = c.n_layers
    value_flops = (2.0 * N * D * D * (L - 1) + 2.0 * N * 3 * D * D * L + 2.0 * E * D * D * L
                   + 2.0 * D * K * nsq + 2.0 * D * D)
    return shapes, value_flops


def message_flops_per_walker(wl):
    """Algorithmic FLOPs of one jet message launch per walker (layer >= 1): for every receiver i,
    node channel c and feature, the sum over the other electrons of w_ij z_j[c] (2 FLOPs each),
    plus the product-rule terms of the coordinate and Laplacian channels."""
    s, c = wl.system, wl.cfg
    N, D, M = s.n_elec, c.width, s.n_nuc
    C = 3 * N + 2
    main = 2.0 * N * (N - 1) * C * D
    prod = (2.0 * N * (N - 1) * 3 * 2 + 2.0 * N * (N - 1) * 8 + 2.0 * N * M * 10) * D
    return main + prod


def wl_edges(wl):
    """Edges per walker: electron pairs (i < j) and electron-nucleus pairs."""
    N, M = wl.system.n_elec, wl.system.n_nuc
    return N * (N - 1) // 2 + N * M


def det_flops_per_walker(wl):
    """Algorithmic FLOPs of the determinant jets per walker: per (p, spin) matrix of size n with
    T = 3N + 1 tangent channels, LU (2n^3/3), inverse (4n^3/3), the tangent products A^-1 dA
    (T 2n^3), their traces and tr((A^-1 dA)^2) (T 2n^2) and tr(A^-1 Lap A) (2n^2)."""
    s, c = wl.system, wl.cfg
    N = s.n_elec
    T = 3 * N + 1
    tot = 0.0
    for n in ((N,) if c.full_det else (s.n_up, s.n_down)):
        if n:
            tot += c.n_det * (2 * n ** 3 / 3 + 4 * n ** 3 / 3 + T * 2 * n ** 3 + T * 2 * n * n + 2 * n * n)
    return tot


def roofline_for(kind, ms, n, wl, chunk, pk, how, alu, steps):
    """Roofline entry of one kernel kind: algorithmic work per launch / average launch time, against
    the bound the kernel runs into (tensor cores for the GEMMs, the CUDA cores' FMA rate for the
    message contraction and the determinant jets, HBM for the streaming kernels)."""
    s, c = wl.system, wl.cfg
    N, D, M = s.n_elec, c.width, s.n_nuc
    C = 3 * N + 2
    E = N * (N - 1) // 2 + N * M
    t = ms / n / 1e3
    bf16 = wl.precision == "bf16"
    shapes, value_flops = gemm_shapes(wl, chunk)
    el = 8 if wl.precision == "fp64" else 4
    base = {"kernel": kind, "avg_launch_ms": ms / n, "launches": n}
    if kind in shapes:
        m, k, n_out = shapes[kind]
        flops = 2.0 * m * k * n_out
        if wl.precision == "fp64":
            peak, bound, src = alu["fp64_tflops"], "alu", "measured FP64 FMA rate (CUDA cores)"
        elif bf16 and kind in ("jet.gemm_update", "jet.gemm_node"):
            peak, bound, src = pk["bf16_tflops_sustained"], "tensor", f"{how} bf16 sustained (cuBLAS loop)"
        else:
            # FP32 operands as three TF32 tensor-core products: TF32 peak (measured bf16 x nominal 1.1/2.25) / 3
            peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0
            bound, src = "tensor", f"{how} bf16 sustained x 1.1/2.25 (TF32) / 3 (3xTF32 split)"
        ach = flops / t / 1e12
        return {**base, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_source": src, "flops_per_launch": flops}
    if kind in ("bwd_gemm", "bwd_reduce"):
        # per launch: the value-only forward GEMM FLOPs of the step's walkers, once per kind and step,
        # spread over the kind's launches
        flops = value_flops * chunk * steps / n
        peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0 if wl.precision != "fp64" else alu["fp64_tflops"]
        ach = flops / t / 1e12
        return {**base, "bound": "tensor" if wl.precision != "fp64" else "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": f"{how} bf16 sustained x 1.1/2.25 / 3 (3xTF32)",
                "flops_per_launch": flops,
                "note": "reverse-pass products of the value-only network (input adjoints for bwd_gemm, weight "
                        "gradients for bwd_reduce), averaged over the kind's launches"}
    if kind == "jet.layer_fused":
        # the update map W_g over every node channel (the S5 GEMM, 2 N C 3D D per walker) as produced on
        # the tensor cores; the electron-electron message contraction (CUDA cores) runs inside the same
        # kernel and is reported beside it
        flops = 2.0 * chunk * N * C * 3 * D * D
        peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0
        ach = flops / t / 1e12
        return {**base, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": LAYER_FUSED_DRAM_BYTES_PER_WALKER * chunk if LAYER_FUSED_DRAM_BYTES_PER_WALKER else None,
                # z read once, the filter jets (w, w', w'') read, the pre-activations written
                "algorithmic_bytes_per_launch": chunk * 4.0 * (2 * N * C * D + wl_edges(wl) * 3 * D),
                "peak_source": f"{how} bf16 sustained x 1.1/2.25 (TF32) / 3 (3xTF32 split)",
                "flops_per_launch": flops, "message_flops_per_launch": message_flops_per_walker(wl) * chunk,
                "message_tflops": message_flops_per_walker(wl) * chunk / t / 1e12,
                "note": "messages, update map and the electron-nucleus part of one layer; FLOPs of the update "
                        "map (the kernel's tensor-core work), averaged over the layer launches"}
    if kind == "jet.messages":
        L = c.n_layers
        flops = message_flops_per_walker(wl) * chunk
        peak = alu["fp32_tflops"] if wl.precision != "fp64" else alu["fp64_tflops"]
        ach = flops / t / 1e12
        byts = (chunk * N * C * D * el * (L - 1) / L) + chunk * E * 3 * D * el + chunk * N * C * 3 * D * (2 if bf16 else el)
        traffic = None
        if wl.name == "n2_fp32" and MSG_DRAM_BYTES_PER_WALKER:
            traffic = MSG_DRAM_BYTES_PER_WALKER * chunk
        elif wl.name == "c4h4_bf16" and MSG_LARGE_DRAM_BYTES_PER_WALKER:
            traffic = MSG_LARGE_DRAM_BYTES_PER_WALKER * chunk
        return {**base, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic, "peak_source": "FMA rate of the CUDA cores measured in this run",
                "flops_per_launch": flops, "bytes_per_launch": byts,
                "traffic_over_bytes": traffic / byts if traffic else None,
                "note": "FLOPs of a layer >= 1 launch (layer 0 has constant node channels and does less)"}
    if kind == "jet.orbital_det":
        flops = det_flops_per_walker(wl) * chunk
        peak = alu["fp32_tflops"] if wl.precision != "fp64" else alu["fp64_tflops"]
        ach = flops / t / 1e12
        return {**base, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_source": "FMA rate of the CUDA cores measured in this run",
                "flops_per_launch": flops,
                "note": "FP64-accurate work: the tangent contractions run in double-float on the FP32 pipes "
                        "(about 20 FP32 operations per algorithmic multiply-add) or on the FP64 pipes"}
    # update: reads the pre-activations and the embeddings, writes the embeddings; edge hidden layer:
    # reads the Gaussian features, writes the hidden jets
    hbm = {"jet.update": 3.0 * chunk * N * C * D * el, "jet.edge_hidden": chunk * E * 3 * (D + 16) * el}
    if kind in hbm:
        byts = hbm[kind]
        ach = byts / t / 1e9
        return {**base, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_source": f"{how} copy bandwidth",
                "bytes_per_launch": byts}
    return None


def profile_case(args):
    import torch

    from paper_2307_14123_gb300 import Ansatz
    from paper_2307_14123_gb300 import fixtures as fx

    wl = fx.workload(args.workload)
    prec = args.profile_precision or wl.precision
    dt = torch.float64 if prec == "fp64" else torch.float32
    h = Ansatz(wl.system, wl.cfg, prec, device="cuda:0")
    theta = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=dt, device="cuda:0")
    r = torch.tensor(fx.init_walkers(wl.system, args.profile_case, wl.walker_seed), dtype=dt, device="cuda:0")
    if args.msg_ib:
        h.set_msg_tile(args.msg_ib)
    if args.profile_op == "grad":
        w = torch.full((args.profile_case,), 1.0 / args.profile_case, dtype=dt, device="cuda:0")
        out = h.grad_logpsi(theta, r, w, 0)
    elif args.profile_op == "mcmc":
        la, _ = h.ansatz_eval(theta, r)
        out = h.mcmc_step(theta, r, la, 1, 0.2, 1, 0)
    else:
        out = h.local_energy(theta, r)[2]
    torch.cuda.synchronize()
    print("profile case done:", args.profile_op, args.profile_case, "walkers", float(out.double().abs().sum()))
    return 0


def natgrad_leg(h, theta, r, wl, args, flush):
    """The natural-gradient direction of one optimisation step on the bench walkers: per-walker
    gradients (grad_logpsi mode 1), clipped-energy weights, then natural_gradient (Gram matrix of
    the centred gradients on the tensor cores, conjugate gradients in FP64)."""
    import torch

    B = r.shape[0]
    _, _, el = h.local_energy(theta, r)
    w, _ = h.vmc_loss_weights(el, 5.0)
    G = h.grad_logpsi(theta, r, mode=1)
    Gc_sq = float(((G.double() - G.double().mean(dim=0)) ** 2).sum())
    lam = 1e-1 * Gc_sq / B / B  # 1e-1 of the mean eigenvalue of Gc Gc^T / B
    h.natural_gradient(G, w, lam, max_iter=500, tol=1e-8)  # warm-up (workspace)
    torch.cuda.synchronize()
    times = {"grad_per_walker": 0.0, "natural_gradient": 0.0}
    reps = 3
    for _ in range(reps):
        flush.fill_(1)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        G = h.grad_logpsi(theta, r, mode=1)
        b.record()
        d, st = h.natural_gradient(G, w, lam, max_iter=500, tol=1e-8)
        c.record()
        torch.cuda.synchronize()
        times["grad_per_walker"] += a.elapsed_time(b) / reps
        times["natural_gradient"] += b.elapsed_time(c) / reps
    st = st.cpu().tolist()
    P = h.P
    gram_flops = 2.0 * B * B * P
    return {"walkers": B, "params": P, "ms_grad_per_walker": times["grad_per_walker"],
            "ms_natural_gradient": times["natural_gradient"], "cg_iterations": st[0], "cg_rel_residual": st[1],
            "damping": "1e-1 x mean eigenvalue of Gc Gc^T / B",
            "gram_fp32_tflops_incl_solve": gram_flops / (times["natural_gradient"] / 1e3) / 1e12,
            "note": "Gram matrix of the centred per-walker gradients (3xTF32 tensor cores, FP32 chunks of 8192 "
                    "parameters added in FP64), conjugate gradients in FP64, delta = Gc^T x"}


def pp_leg(h, theta, r, wl, flush, B=512):
    """Local and non-local pseudopotential energies (synthetic coefficients, l_max 2, on both
    nuclei) for B of the bench walkers: B * N * 2 * 12 value-only psi evaluations per call."""
    import torch

    from paper_2307_14123_gb300 import fixtures as fx

    rr = r[:B].contiguous()
    la, sg = h.ansatz_eval(theta, rr)
    pps = [(0, fx.synthetic_pseudopotential(2, seed=5)), (1, fx.synthetic_pseudopotential(2, seed=6))]
    rot = torch.tensor(fx.random_rotations(B, 7), dtype=rr.dtype, device=rr.device)
    h.pseudopotential_energy(theta, rr, pps, rot, la, sg)
    torch.cuda.synchronize()
    tot, reps = 0.0, 3
    for _ in range(reps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        h.pseudopotential_energy(theta, rr, pps, rot, la, sg)
        b.record()
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    ms = tot / reps
    n_eval = B * wl.system.n_elec * len(pps) * 12
    return {"walkers": B, "psi_evaluations": n_eval, "ms_per_call": ms,
            "psi_evaluations_per_s": n_eval / (ms / 1e3),
            "note": "12-point icosahedral quadrature, every electron around both nuclei, synthetic coefficients"}


def graph_kernel_count(fn):
    """Kernel launches of one call of fn: the kernel nodes of a CUDA graph captured from it (the
    capture enqueues nothing; memset and copy nodes are not counted)."""
    import ctypes

    import torch

    g = torch.cuda.CUDAGraph(keep_graph=True)
    with torch.cuda.graph(g):
        fn()
    cu = ctypes.CDLL("libcuda.so.1")
    handle = ctypes.c_void_p(g.raw_cuda_graph())
    n = ctypes.c_size_t(0)
    if cu.cuGraphGetNodes(handle, None, ctypes.byref(n)) != 0:
        raise RuntimeError("cuGraphGetNodes failed")
    nodes = (ctypes.c_void_p * max(n.value, 1))()
    if cu.cuGraphGetNodes(handle, nodes, ctypes.byref(n)) != 0:
        raise RuntimeError("cuGraphGetNodes failed")
    kind, kernels = ctypes.c_int(), 0
    for i in range(n.value):
        if cu.cuGraphNodeGetType(ctypes.c_void_p(nodes[i]), ctypes.byref(kind)) != 0:
            raise RuntimeError("cuGraphNodeGetType failed")
        kernels += kind.value == 0  # CU_GRAPH_NODE_TYPE_KERNEL
    del g
    return kernels


def ansatz_variants_leg(h, theta, r, wl, flush, reps=5):
    """Local energies of the ansatz variants on the bench walkers, each timed like the base
    (spin-factorised determinants, fixed Gaussian edge features, spin initial embeddings): the
    full determinant (Eq. 22), iterated edge embeddings (Eq. 16, second case), both (the
    PauliNet2-style ansatz), and initial embeddings from the electron-nucleus difference vectors
    (Eq. 13, second case)."""
    import dataclasses

    import torch

    from paper_2307_14123_gb300 import Ansatz
    from paper_2307_14123_gb300 import fixtures as fx

    def timed(hh, th):
        hh.local_energy(th, r)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            hh.local_energy(th, r)
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    B = r.shape[0]
    ms_base = timed(h, theta)
    out = {"base": {"value": B / (ms_base / 1e3), "unit": UNIT, "ms_per_call": ms_base, "params": h.P}}
    for name, kw in (("full_determinant", {"full_det": 1}), ("edge_update", {"edge_update": 1}),
                     ("full_determinant+edge_update", {"full_det": 1, "edge_update": 1}),
                     ("electron_nucleus_init", {"el_init": 1})):
        cfg = dataclasses.replace(wl.cfg, **kw)
        hv = Ansatz(wl.system, cfg, wl.precision, device=r.device)
        th = torch.tensor(fx.init_params(wl.system, cfg, wl.param_seed), dtype=theta.dtype, device=r.device)
        ms = timed(hv, th)
        out[name] = {"value": B / (ms / 1e3), "unit": UNIT, "ms_per_call": ms, "params": hv.P,
                     "cost_vs_base": ms / ms_base}
        del hv
    out["note"] = (f"{wl.system.name} {wl.precision.upper()}, {B} walkers, local_energy calls, L2 flushed "
                   "before each; full determinant: one N x N matrix per p instead of two spin blocks")
    return out


def bf16_leg(h, theta, r, wl, flush, reps=5):
    """BF16 mode against FP32: local_energy on the bench walkers in both modes (same timing as the
    base), with the paired change of the mean local energy; and the paired BF16 - FP32 mean shift on
    a trained low-variance state (LiH, width 64, two layers, one determinant: 200 natural-gradient
    steps in FP32 from random initialisation, 65,536 walkers after 200 Metropolis sweeps)."""
    import numpy as np
    import torch

    from paper_2307_14123_gb300 import Ansatz, vmc_train_step
    from paper_2307_14123_gb300 import fixtures as fx

    dev = r.device
    out = {}

    def timed(hh):
        res = hh.local_energy(theta, r)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            hh.local_energy(theta, r)
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps, res[2].double()

    h32 = Ansatz(wl.system, wl.cfg, "fp32", device=dev)
    h16 = Ansatz(wl.system, wl.cfg, "bf16", device=dev)
    ms32, e32 = timed(h32)
    ms16, e16 = timed(h16)
    d = (e16 - e32)[torch.isfinite(e16 - e32)]
    B = r.shape[0]
    out["bench_walkers"] = {"fp32_ms_per_call": ms32, "bf16_ms_per_call": ms16, "bf16_speedup": ms32 / ms16,
                            "fp32_value": B / (ms32 / 1e3), "bf16_value": B / (ms16 / 1e3), "unit": UNIT,
                            "mean_dE_bf16_minus_fp32": float(d.mean()),
                            "stderr": float(d.std() / max(1, d.numel()) ** 0.5),
                            "note": "random-initialised ansatz; both modes run the fused layer kernel (FP32: "
                                    "3 x TF32 update-map products; BF16: BF16 operands of W_g's "
                                    "electron-electron blocks, FP32 accumulation); node maps on 3 x TF32"}
    del h32, h16
    system = fx.molecule("LiH")
    cfg = fx.AnsatzCfg(64, 2, 1)
    t32 = Ansatz(system, cfg, "fp32", device=dev)
    t16 = Ansatz(system, cfg, "bf16", device=dev)
    th = torch.tensor(fx.init_params(system, cfg, 3), dtype=torch.float32, device=dev)
    rt = torch.tensor(fx.init_walkers(system, 1024, 3), dtype=torch.float32, device=dev)
    la, _ = t32.ansatz_eval(th, rt)
    t32.mcmc_step(th, rt, la, 50, 0.2, 9, 0)
    for t in range(200):
        vmc_train_step(t32, th, rt, la, lr=0.2, damping=-0.1, max_norm=0.3, seed=1, step_counter=50 + t)
    Bt = 65536
    rr = torch.tensor(fx.init_walkers(system, Bt, 21), dtype=torch.float32, device=dev)
    la2, _ = t32.ansatz_eval(th, rr)
    t32.mcmc_step(th, rr, la2, 200, 0.2, 21, 0)
    a32 = t32.local_energy(th, rr)[2].double().cpu().numpy()
    a16 = t16.local_energy(th, rr)[2].double().cpu().numpy()
    dd = a16 - a32
    out["trained_lih"] = {"walkers": Bt, "mean_e_loc_fp32": float(a32.mean()), "variance_fp32": float(a32.var()),
                          "mean_dE_bf16_minus_fp32": float(dd.mean()), "stderr": float(dd.std() / np.sqrt(Bt)),
                          "variance_change_rel": float(a16.var() / a32.var() - 1),
                          "median_abs_dE": float(np.median(np.abs(dd)))}
    return out


def training_leg(dev, steps=60):
    """VMC training end to end in the library (vmc_train_step: Metropolis sweep, local energies,
    clipped-energy weights, per-walker gradients, natural gradient, parameter update) on LiH in
    FP32 from random initialisation: mean local energy per block of 10 steps and time per step."""
    import torch

    from paper_2307_14123_gb300 import Ansatz, vmc_train_step
    from paper_2307_14123_gb300 import fixtures as fx

    wl = fx.workload("lih_fp64")
    h = Ansatz(wl.system, wl.cfg, "fp32", device=dev)
    th = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=torch.float32, device=dev)
    B = 1024
    r = torch.tensor(fx.init_walkers(wl.system, B, wl.walker_seed), dtype=torch.float32, device=dev)
    la, _ = h.ansatz_eval(th, r)
    h.mcmc_step(th, r, la, 50, 0.2, 9, 0)  # equilibration of the walkers
    sums = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for t in range(steps):
        sums.append(vmc_train_step(h, th, r, la, lr=0.2, damping=-0.1, max_norm=0.3, seed=1,
                                   step_counter=50 + t)["e_sum2"])
    b.record()
    torch.cuda.synchronize()
    e = [float(x[0]) / B for x in sums]
    return {"molecule": "LiH", "walkers": B, "steps": steps, "ms_per_step": a.elapsed_time(b) / steps,
            "mean_energy_per_10_steps": [sum(e[i:i + 10]) / 10 for i in range(0, steps, 10)],
            "settings": "lr 0.2, step-length limit 0.3, damping 0.1 x mean eigenvalue, 50 equilibration sweeps",
            "note": "random-initialised ansatz; the exact non-relativistic LiH energy is about -8.07 Ha"}


def batch_leg(args, dev, flush):
    """The uneven-molecule batch (H2O, NH3, C2H4, C6H6; 8192/8192/4096/2048 walkers): local
    energies of all molecules in one grouped call per step, after the autotuner picked its
    tile shapes, against the same molecules run one after another through single-molecule
    handles (plain FP32 path); then the batch's whole VMC step as one CUDA graph."""
    import torch

    from paper_2307_14123_gb300 import Ansatz, AnsatzBatch
    from paper_2307_14123_gb300 import fixtures as fx

    def timed(fn, steps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    out = {}
    steps = max(3, min(args.steps, 10))
    for prec in ("fp32", "bf16"):
        wls = fx.batch_workload("mixed_" + prec)
        batch = AnsatzBatch([w.system for w in wls], [w.cfg for w in wls], prec, device=dev)
        th = [torch.tensor(fx.init_params(w.system, w.cfg, w.param_seed), dtype=torch.float32, device=dev)
              for w in wls]
        r = [torch.tensor(fx.init_walkers(w.system, w.B, w.walker_seed), dtype=torch.float32, device=dev)
             for w in wls]
        walkers = sum(w.B for w in wls)
        tune_ms, rounds, ib = batch.autotune(th, r)
        res = {}
        ms_b = timed(lambda: res.__setitem__("el", batch.local_energy(th, r)[2]), steps)
        entry = {"value": walkers / (ms_b / 1e3), "unit": UNIT, "ms_per_call": ms_b, "walkers": walkers,
                 "tuning": dict(batch.tile_set(), autotune_ms=tune_ms)}
        if prec == "fp32":
            singles = [Ansatz(w.system, w.cfg, "fp32", device=dev) for w in wls]
            ms_p = timed(lambda: [h.local_energy(th[k], r[k]) for k, h in enumerate(singles)], steps)
            entry["plain_fp32_one_by_one"] = {"value": walkers / (ms_p / 1e3), "ms_per_call": ms_p}
            entry["speedup_vs_plain"] = ms_p / ms_b
            el32 = [e.double() for e in res["el"]]
            out["fp32"] = entry
            del singles
            # the batch's VMC step (Metropolis sweep, local energies, loss weights, gradients) as one graph
            la, _ = batch.ansatz_eval(th, r)
            ctr = torch.zeros(1, dtype=torch.int64, device=dev)

            def vstep():
                batch.mcmc_step(th, r, la, 1, 0.2, 4, ctr)
                _, _, el = batch.local_energy(th, r)
                w, _ = batch.vmc_loss_weights(el, 5.0)
                return batch.grad_logpsi(th, r, w)

            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                vstep()
            torch.cuda.current_stream().wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                vstep()
            ms_g = timed(g.replay, steps)
            entry["vmc_step_graph"] = {"value": walkers / (ms_g / 1e3), "unit": UNIT, "ms_per_step": ms_g,
                                       "step": "mcmc_step_multi + local_energy_multi + vmc_loss_weights_multi + "
                                               "grad_logpsi_multi, captured once, replayed"}
            del g
        else:
            # BF16 embedding GEMMs against the FP32 batch on the same walkers: change of each
            # molecule's mean local energy with the standard error of the per-walker differences
            el16 = [e.double() for e in res["el"]]
            dev_e = []
            for k, w in enumerate(wls):
                d = el16[k] - el32[k]
                fin = torch.isfinite(d)
                d = d[fin]
                dev_e.append({"molecule": w.system.name, "mean_dE": float(d.mean()),
                              "stderr": float(d.std() / max(1, d.numel()) ** 0.5)})
            entry["mean_energy_change_vs_fp32"] = dev_e
            entry["speedup_vs_fp32_batch"] = out["fp32"]["ms_per_call"] / ms_b
            entry["speedup_vs_plain_fp32"] = out["fp32"]["plain_fp32_one_by_one"]["ms_per_call"] / ms_b
            out["bf16"] = entry
        del batch
        torch.cuda.empty_cache()
    out["workload"] = ("H2O 10e / NH3 10e / C2H4 16e / C6H6 42e, D=128, L=3, K=8, "
                       "8192/8192/4096/2048 walkers, local energies of all molecules per call")
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2307_14123_gb300 import Ansatz
    from paper_2307_14123_gb300 import fixtures as fx
    from paper_2307_14123_gb300.binding import DQError

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    wl = fx.workload(args.workload)
    B = wl.B
    dt = torch.float64 if wl.precision == "fp64" else torch.float32
    h = Ansatz(wl.system, wl.cfg, wl.precision, device=dev)
    theta = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=dt, device=dev)
    r0 = fx.init_walkers(wl.system, B, wl.walker_seed, walker_offset=rank * B)
    r = torch.tensor(r0, dtype=dt, device=dev)
    logabs, _ = h.ansatz_eval(theta, r)
    # tile shapes (message register tile, walker chunk) timed on these walkers before the timed region
    tuning = None
    if wl.precision != "fp64" and not args.no_autotune:
        t_ms, t_chunk, t_ib = h.autotune(theta, r)
        tuning = dict(h.tile_set(), local_energy_ms=t_ms)
    elif wl.precision != "fp64":
        tuning = dict(h.tile_set(), autotuned=False)
    step_size = wl.extra.get("step_size", 0.2)
    try:
        h.grad_logpsi(theta, r[:1], torch.ones(1, dtype=dt, device=dev), 0)
        with_grad = True
    except DQError:
        with_grad = False
    counter = [0]

    def step(th, rr, la):
        h.mcmc_step(th, rr, la, 1, step_size, wl.walker_seed, counter[0])
        counter[0] += 1
        la2, _, el, e2 = h.local_energy(th, rr, sums=True)
        w, stats = h.vmc_loss_weights(el, 5.0)
        g = h.grad_logpsi(th, rr, w, 0) if with_grad else None
        return el, e2, g

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # FMA rates of the CUDA cores on this GPU (the bound of the kernels that run on them), with the
    # SM clock sampled while the probes run; no GPU setting is changed
    from paper_2307_14123_gb300.binding import fma_rate
    alu_clk = ClockSampler(local)
    alu_clk.start()
    alu = {"fp32_tflops": fma_rate("fp32", dev), "fp64_tflops": fma_rate("fp64", dev)}
    alu["clocks"] = alu_clk.stop()
    alu["how"] = ("dq_fma_rate_probe: 1216 blocks x 256 threads, 8 independent FMA chains per thread, best of 5 "
                  "launches timed with CUDA events")
    for _ in range(args.warmup):
        step(theta, r, logabs)
    torch.cuda.synchronize()
    h.fp64_matrix_count()  # cleared: the timed steps' count is read after them

    h.profile(True)
    h.profile_reset()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(theta, r, logabs)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    h.profile(False)
    n_fp64 = h.fp64_matrix_count()
    n_mat_step = 2 * B * wl.cfg.n_det * 2  # the sampler's value-only forward and the jets forward
    fp64_dets = {"per_step": n_fp64 / args.steps, "matrices_per_step": n_mat_step,
                 "fraction": n_fp64 / args.steps / n_mat_step,
                 "note": "determinant matrices factorised in FP64 (ill-conditioned ones) by the timed steps, "
                         "both forwards of a step"}
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    prof = h.profile_read()
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = B * world * args.steps / (total_ms / 1e3)

    # local_energy alone (same timed-kernel view, from the profile)
    jet_ms = sum(ms for k, (ms, n) in prof.items() if k.startswith("jet.") or k == "esum")
    launch_sites = sum(n for _, (ms, n) in prof.items())
    # kernels of one step: the kernel nodes of a CUDA-graph capture of the same step (a launch
    # site of the library may launch several kernels, e.g. a split reduction and its sum)
    kernels_per_step = graph_kernel_count(lambda: step(theta, r, logabs))
    launches = kernels_per_step * args.steps
    gpu_time_ms = sum(ms for _, (ms, n) in prof.items())

    # roofline of the dominant kernel (and of the other main kernels)
    pk, how = peaks()
    chunk = min(B, h.max_chunk())
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    roof = None
    others = []
    for kind in ("jet.layer_fused", "jet.messages", "jet.gemm_update", "jet.gemm_edge", "jet.gemm_node",
                 "jet.gemm_orbital", "jet.orbital_det", "jet.update", "jet.edge_hidden", "bwd_gemm", "bwd_reduce"):
        if kind in prof:
            e = roofline_for(kind, prof[kind][0], prof[kind][1], wl, chunk, pk, how, alu, args.steps)
            if e:
                e["share_of_gpu_time"] = prof[kind][0] / gpu_time_ms
                others.append(e)
    if dom is not None:
        roof = roofline_for(dom, prof[dom][0], prof[dom][1], wl, chunk, pk, how, alu, args.steps)
        if roof:
            roof["share_of_gpu_time"] = prof[dom][0] / gpu_time_ms
        else:
            roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                    "traffic": None, "note": "no roofline formula for this kernel kind",
                    "share_of_gpu_time": prof[dom][0] / gpu_time_ms}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        th_h = theta.cpu().pin_memory()
        r_h = r.cpu().pin_memory()
        la_h = logabs.cpu().pin_memory()
        el_h = torch.empty(B, dtype=dt).pin_memory()
        g_h = torch.empty(h.P, dtype=dt).pin_memory() if with_grad else None
        th_d, r_d, la_d = torch.empty_like(theta), torch.empty_like(r), torch.empty_like(logabs)
        h2d = th_h.numel() * th_h.element_size() + r_h.numel() * r_h.element_size() + la_h.numel() * la_h.element_size()
        d2h = r_h.numel() * r_h.element_size() + la_h.numel() * la_h.element_size() + el_h.numel() * el_h.element_size()
        if with_grad:
            d2h += g_h.numel() * g_h.element_size()

        def e2e_step():
            th_d.copy_(th_h, non_blocking=True)
            r_d.copy_(r_h, non_blocking=True)
            la_d.copy_(la_h, non_blocking=True)
            el, _, g = step(th_d, r_d, la_d)
            r_h.copy_(r_d, non_blocking=True)
            la_h.copy_(la_d, non_blocking=True)
            el_h.copy_(el, non_blocking=True)
            if g is not None:
                g_h.copy_(g, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        # same conditions as the device-timed steps: L2 flushed before every step (outside the
        # timed interval), the library's per-launch events on
        h.profile_reset()
        h.profile(True)
        ev2 = []
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            e2e_step()
            b.record()
            ev2.append((a, b))
        torch.cuda.synchronize()
        h.profile(False)
        t2 = torch.tensor([sum(a.elapsed_time(b) for a, b in ev2)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t2, op=dist.ReduceOp.MAX)
        e2e = {"value": B * world * args.steps / (float(t2.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "each step: parameters, positions and log|psi| copied from pinned host memory (one "
                       "cudaMemcpyAsync per array), the step through the public API, positions, log|psi|, "
                       "E_loc and the gradient copied back; L2 flushed before every step and the library's "
                       "per-launch events on, as for value"}

    # the same step captured as one CUDA graph (step counter on the device) and replayed
    graph = None
    if not args.no_graph:
        ctr = torch.tensor([counter[0]], dtype=torch.int64, device=dev)

        def gstep(th, rr, la):
            h.mcmc_step(th, rr, la, 1, step_size, wl.walker_seed, ctr)
            la2, _, el, e2 = h.local_energy(th, rr, sums=True)
            w, stats = h.vmc_loss_weights(el, 5.0)
            g = h.grad_logpsi(th, rr, w, 0) if with_grad else None
            return el, e2, g

        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            gstep(theta, r, logabs)
        torch.cuda.current_stream().wait_stream(side)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            gstep(theta, r, logabs)
        for _ in range(args.warmup):
            cg.replay()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        gev = []
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            cg.replay()
            b.record()
            gev.append((a, b))
        torch.cuda.synchronize()
        t3 = torch.tensor([sum(a.elapsed_time(b) for a, b in gev)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t3, op=dist.ReduceOp.MAX)
        gms = float(t3.item())
        graph = {"value": B * world * args.steps / (gms / 1e3), "unit": UNIT, "ms_per_step": gms / args.steps,
                 "note": "the timed step replayed as one CUDA graph (Metropolis step counter on the device), "
                         "L2 flushed before every replay"}
        del cg

    # the VMC step with the Langevin sampler in place of the Metropolis one: the proposal's
    # forward (value, drift, Laplacian) also gives E_loc at the accepted positions, so the
    # step is mala_step + vmc_loss_weights + grad_logpsi
    langevin = None
    if not args.no_mala:
        tau = args.mala_tau
        r_m, la_m = r.clone(), torch.empty_like(logabs)
        g_m, e_m = torch.empty_like(r), torch.empty_like(logabs)
        h.mala_step(theta, r_m, la_m, g_m, n_steps=0, tau=tau, grad_valid=False, e_loc=e_m)
        mctr = torch.zeros(1, dtype=torch.int64, device=dev)

        def mstep():
            n = h.mala_step(theta, r_m, la_m, g_m, 1, tau, wl.walker_seed + 1, mctr, e_loc=e_m)
            w, stats = h.vmc_loss_weights(e_m, 5.0)
            g = h.grad_logpsi(theta, r_m, w, 0) if with_grad else None
            return n

        for _ in range(args.warmup):
            mstep()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        mev, n_acc = [], torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            n = mstep()
            b.record()
            n_acc += n
            mev.append((a, b))
        torch.cuda.synchronize()
        t4 = torch.tensor([sum(a.elapsed_time(b) for a, b in mev)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t4, op=dist.ReduceOp.MAX)
        mms = float(t4.item())
        langevin = {"value": B * world * args.steps / (mms / 1e3), "unit": UNIT, "ms_per_step": mms / args.steps,
                    "tau": tau, "acceptance": int(n_acc.item()) / (B * args.steps),
                    "step": "mala_step(1 Langevin sweep, E_loc carried) + vmc_loss_weights"
                            + (" + grad_logpsi(weighted)" if with_grad else ""),
                    "note": "same workload, Langevin sampler (Sec. 5) instead of random-walk Metropolis; "
                            "L2 flushed before every step"}

    # the same Metropolis chain with E_loc carried: proposals evaluated by the jets forward
    # (mcmc_step_eloc), one forward per step instead of the value-only forward + local_energy
    metro_eloc = None
    if not args.no_mala:
        r_e = r.clone()
        la_e, _, e_e = h.local_energy(theta, r_e)
        ectr = torch.zeros(1, dtype=torch.int64, device=dev)

        def estep():
            n = h.mcmc_step_eloc(theta, r_e, la_e, e_e, 1, step_size, wl.walker_seed, ectr)
            w, stats = h.vmc_loss_weights(e_e, 5.0)
            g = h.grad_logpsi(theta, r_e, w, 0) if with_grad else None
            return n

        for _ in range(args.warmup):
            estep()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        eev, e_acc = [], torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            n = estep()
            b.record()
            e_acc += n
            eev.append((a, b))
        torch.cuda.synchronize()
        t5 = torch.tensor([sum(a.elapsed_time(b) for a, b in eev)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t5, op=dist.ReduceOp.MAX)
        ems = float(t5.item())
        metro_eloc = {"value": B * world * args.steps / (ems / 1e3), "unit": UNIT, "ms_per_step": ems / args.steps,
                      "acceptance": int(e_acc.item()) / (B * args.steps),
                      "step": "mcmc_step_eloc(1 Metropolis sweep, proposals through the jets forward, E_loc "
                              "carried) + vmc_loss_weights" + (" + grad_logpsi(weighted)" if with_grad else ""),
                      "note": "the headline step's Metropolis chain and outputs with one forward per walker; "
                              "L2 flushed before every step"}

    natgrad = natgrad_leg(h, theta, r, wl, args, flush) if (world == 1 and with_grad and not args.no_natgrad) else None
    batched = batch_leg(args, dev, flush) if (world == 1 and not args.no_batch) else None
    training = training_leg(dev) if (world == 1 and not args.no_natgrad) else None
    pseudo = pp_leg(h, theta, r, wl, flush) if (world == 1 and not args.no_pp) else None
    variants = ansatz_variants_leg(h, theta, r, wl, flush) if (world == 1 and not args.no_pp) else None
    bf16 = bf16_leg(h, theta, r, wl, flush) if (world == 1 and not args.no_pp and wl.precision == "fp32") else None

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, parity = oracle_leg(h, wl, args.cpu_seconds, dev, with_grad)

    if rank == 0:
        step_desc = "mcmc_step(1 sweep) + local_energy + vmc_loss_weights" + (" + grad_logpsi(weighted)" if with_grad
                                                                             else " (grad_logpsi not built)")
        cfg = workload_config(wl, world)
        cfg.update({"step": step_desc, "l2": "flushed before every timed step (256 MB write)", "tuning": tuning})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16+f32"}[wl.precision],
                "data": "synthetic (seeded walkers and random-init weights)", "config": cfg,
                "roofline": roof, "roofline_main_kernels": others, "alu_peaks": alu, "cpu_baseline": cpu,
                "parity_vs_oracle": parity, "e2e": e2e,
                "cuda_graph": graph,
                "langevin_sampler": langevin,
                "metropolis_eloc_carried": metro_eloc,
                "batched_molecules": batched,
                "natural_gradient": natgrad,
                "vmc_training": training,
                "pseudopotential": pseudo,
                "ansatz_variants": variants,
                "bf16_mode": bf16,
                "fp64_determinants": fp64_dets,
                "gpu_launches": launches,
                "gpu_kernels_per_step": kernels_per_step,
                "gpu_launch_sites": launch_sites,
                "clocks": clk,
                "local_energy_only": {"value": B * world * args.steps / (jet_ms / 1e3) if jet_ms else None,
                                      "unit": UNIT, "note": "sum of the local_energy kernels' device time"},
                "kernels_ms_per_step": {k: round(ms / args.steps, 4) for k, (ms, n) in
                                        sorted(prof.items(), key=lambda kv: -kv[1][0])},
                "peaks": how}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
