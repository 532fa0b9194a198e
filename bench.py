#!/usr/bin/env python
"""Benchmark of the ACSE hot path on GB300 (one JSON line on rank 0).

A step is one Euler step of Eq. (update) through the C ABI (`acse_step`): the residual A at D
(1-RDM, M, pair-pair and particle-hole GEMMs, B and G assembly, FP64 norm), the update
U = 1/2 G(A) with the same reconstruction, D <- D + eps U and the FP64 energy.  The workload is
the r = 48, N = 20, CAS(8e,8o) system (synthetic integrals, seed 0).  The metric is ACSE
residual evaluations per second over all ranks, one evaluation being one contraction pass G(W)
with the reconstructed 3-RDM (the residual G(K/2), or the update's G(A), the same contraction with
another W): a step is two evaluations (its axpy and energy are not counted).  TFLOP/s counts the
O(r^6) GEMM work, 2 M N K summed over the GEMMs (32 r^6 per contraction pass).

--impl reference times the FP64 numpy oracle on the host cores instead (rank 0 only): one full
oracle residual evaluation of the same workload per step.
Multi-GPU: independent replicas (one problem per rank, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# measured on this machine's GB300 by `python bench.py --peaks` (torch.matmul, best of 5-10):
# cuBLAS DGEMM 8192^3 1.10 TFLOP/s, TF32 1041 TFLOP/s; used where MEASURED_PEAKS.json has no entry
FP64_PEAK_TFLOPS = 1.10
TF32_PEAK_TFLOPS = 1041.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=None, choices=["fp64", "bf16x3", "tf32", "tf32x3", "ozaki"])
    ap.add_argument("--recon", default="V", choices=["V", "NY"], help="3-RDM reconstruction")
    ap.add_argument("--singlet", action="store_true",
                    help="spin-flip specialisation of the split path (closed-shell workloads only)")
    ap.add_argument("--r", type=int, default=48, help="orbitals (48: the CAS(8e,8o) workload)")
    ap.add_argument("--eps", type=float, default=None,
                    help="Euler step; default 1e-4 for r >= 32 (1e-3 diverges there), else the paper's 1e-3")
    ap.add_argument("--reset-every", type=int, default=200,
                    help="copy D_0 back into D every this many steps (keeps long runs on the stable stretch)")
    ap.add_argument("--sustain-s", type=float, default=1.5,
                    help="seconds of untimed steps before the timed region, sampled for the clock record")
    ap.add_argument("--gemm-tile", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core GEMM tiling: 0 default, 1 one SM per tile, 2 CTA pairs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--peaks", action="store_true", help="measure FP64/TF32/BF16 matmul peaks and exit")
    ap.add_argument("--batch", action="store_true",
                    help="time the 16-instance batch (r = 12..40, CAS(4e,4o) ground + excited) instead")
    ap.add_argument("--time-to-e", action="store_true",
                    help="time to a converged energy (Methods stopping rule, line search) per precision and "
                         "schedule, then per-iteration errors of fixed steps, against FP64")
    ap.add_argument("--cap", type=int, default=100, help="step cap of --time-to-e")
    ap.add_argument("--adjoint", action="store_true",
                    help="adjoint cost relative to the forward steps (FP64 and Ozaki, r = 32 CAS(6e,6o), 4 steps)")
    return ap.parse_args()


def default_prec():
    # the tensor-core path when this build provides it, else FP64
    try:
        from paper_2604_02550_gb300 import _lib
        return "bf16x3" if getattr(_lib, "HAS_TC", True) else "fp64"
    except Exception:
        return "fp64"


def workload(r, seed=0):
    import acse_inputs as I
    if r == 48:
        return I.config_problem(3, seed)
    if r == 24:
        return I.config_problem(2, seed)
    if r == 32:
        return I.config_problem(5, seed)
    # other sizes: CAS(4e,4o) above a core, N = r/2 rounded to even
    n = max(6, (r // 2) & ~1)
    nc = (n - 4) // 2
    return I.make_problem(r, n, seed, "cas", core=range(nc), active=range(nc, nc + 4), nelecas=4,
                          name=f"cas44_r{r}")


def gemm_traffic(prec):
    """DRAM bytes of one GEMM launch from profiles/gemm_tc_traffic.txt (an ncu capture), or None when
    the kernel source has changed since that capture or the precision differs."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "gemm_tc_traffic.txt")
    if prec != "bf16x3" or not os.path.exists(path):
        return None
    kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
    src = os.path.join(ROOT, "paper_2604_02550_gb300", "csrc", "gemm_tc.cu")
    if hashlib.sha1(open(src, "rb").read()).hexdigest() != kv.get("gemm_tc_sha1"):
        return None
    return float(kv["traffic_bytes"])


OZ_SLICES = 8   # default slices of ACSE_OZAKI
# moduli of the modular Ozaki GEMM, largest first; a context uses the least T whose product covers
# 4 Kmax 2^(2 min(6S, 53)), Kmax = 2 r^2 its longest contraction
OZ_MODULI = (127, 125, 123, 121, 119, 113, 109, 107, 103, 101, 97, 89, 83, 79, 73, 71, 67, 61, 59)


def oz_moduli_count(S, Kmax):
    need, P, T = Kmax << (2 * min(6 * S, 53) + 2), 1, 0
    while T < len(OZ_MODULI) and P < need:
        P *= OZ_MODULI[T]
        T += 1
    return T


def flops_per_pass(r, packed=False, singlet=False):
    """2 M N K over the O(r^6) GEMMs of one contraction pass G(W):
    pair-pair: 3 spin sectors x ([M; D] (2 r^2 rows) x r^2 x r^2); particle-hole: one
    (2r^2)^3 diagonal-sector GEMM and two (r^2)^3 spin-flip GEMMs  ->  32 r^6.
    packed=True counts the plan the tensor-core path runs: the same-spin pair GEMMs on pairs i < j
    only (P = r(r-1)/2: [M; D] 2P rows x P columns x P K each).  singlet=True (spin-flip
    specialisation) drops the bb pair GEMM, the beta-led rows of the diagonal particle-hole GEMM
    and the second spin-flip GEMM."""
    R2 = r * r
    if not packed:
        return 2 * (3 * (2 * R2) * R2 * R2 + (2 * R2) ** 3 + 2 * R2 ** 3)
    P = r * (r - 1) // 2
    if singlet:
        return 2 * ((2 * P) * P * P + (2 * R2) * R2 * R2 + R2 * (2 * R2) * (2 * R2) + R2 ** 3)
    return 2 * (2 * (2 * P) * P * P + (2 * R2) * R2 * R2 + (2 * R2) ** 3 + 2 * R2 ** 3)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, dist=None, device="cuda"):
    """The slowest rank's timed-region length (ms): an all-reduce MAX when a process group is up."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    return float(t)


def whole_job_rate(units_per_rank, world, ms_max):
    """Units per second over all ranks (weak scaling: every rank processes units_per_rank)."""
    return world * units_per_rank / (ms_max / 1e3)


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


EVALS_PER_STEP = 2     # contraction passes of one acse_step: the residual and the update


def cpu_oracle_timing(p, n_evals=1):
    """The FP64 oracle (spin-orbital numpy, all host cores) on `n_evals` residual evaluations."""
    import numpy as np
    from oracle import acse_oracle as O
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    D = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    t0 = time.perf_counter()
    for _ in range(n_evals):
        A = O.residual(K, D, p.N)
    dt = time.perf_counter() - t0
    del A
    return n_evals / dt, dt, os.cpu_count()


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: each step one full oracle residual evaluation of the workload
    (about 23 s at r = 48 on a 16-core Grace host), warm-up steps the same."""
    if rank != 0:
        return
    from oracle import acse_oracle as O
    p = workload(args.r)
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    D = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    for _ in range(args.warmup):
        O.residual(K, D, p.N)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        A = O.residual(K, D, p.N)
        times.append(time.perf_counter() - t0)
        del A
    total = sum(times)
    val = args.steps / total
    sample = f"per step one full FP64 oracle residual evaluation of {p.name} ({total / args.steps:.2f} s each)"
    line = {"metric": "acse_residual_evals_per_s", "value": val, "unit": "residual evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": p.name, "r": p.r, "N": p.N, "prec": "fp64 (numpy oracle, spin-orbital basis)",
                       "step": "one residual evaluation G(K/2)"},
            "cpu_baseline": {"kind": "oracle", "value": val, "unit": "residual evals/s", "cores": os.cpu_count(),
                             "sample": sample},
            "e2e": {"value": val, "unit": "residual evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_peaks():
    import torch
    out = {}

    def mm(dtype, n, iters, tf32=False):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(3):
            a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(iters):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return 2 * n ** 3 / best / 1e12

    out["fp64_tflops"] = mm(torch.float64, 8192, 5)
    out["tf32_tflops"] = mm(torch.float32, 8192, 10, tf32=True)
    out["fp32_simt_tflops"] = mm(torch.float32, 8192, 5)
    out["bf16_tflops"] = mm(torch.bfloat16, 8192, 10)
    out["how"] = "torch.matmul n=8192, best of 5-10 after 3 warm-up calls, CUDA events"
    print(json.dumps(out), flush=True)


def run_batch(args, rank, world):
    """The 16-instance batch: graph-replayed steps, one grouped GEMM launch per pass."""
    import numpy as np
    import torch
    import acse_inputs as I
    from paper_2604_02550_gb300 import _lib
    prec = args.prec or default_prec()
    probs = I.batch_problems(seed=100 * rank)
    eps = args.eps if args.eps is not None else 1e-4
    b = _lib.acse_batch_create(probs, prec)
    for i, p in enumerate(probs):
        _lib.acse_batch_set_D(b, i, p.Daa, p.Dab, p.Dbb, eps)
    _lib.acse_batch_run(b, len(probs), args.warmup, stop_rule=False)
    for i, p in enumerate(probs):
        _lib.acse_batch_set_D(b, i, p.Daa, p.Dab, p.Dbb, eps)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    time.sleep(0.3)
    _, _, l0 = _lib.acse_batch_info(b)
    t0 = time.perf_counter()
    E, N2, S, R = _lib.acse_batch_run(b, len(probs), args.steps, stop_rule=False)
    dt = time.perf_counter() - t0
    clocks = sampler.stop()
    tune, split, launches = _lib.acse_batch_info(b)
    _lib.acse_batch_destroy(b)
    fl = sum(2 * flops_per_pass(p.r, packed=prec != "fp64") for p in probs)
    line = {"metric": "acse_residual_evals_per_s", "value": world * EVALS_PER_STEP * len(probs) * args.steps / dt,
            "unit": "residual evals/s", "evals_per_step": EVALS_PER_STEP * len(probs),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else prec, "data": "synthetic",
            "config": {"workload": "batch16_r12-40_cas44", "instances": len(probs), "prec": prec, "eps": eps,
                       "step": "one graph replay: every instance's residual + update + axpy + energy (two "
                               "residual evaluations per instance)",
                       "tile_choice": tune, "split_r2": split},
            "tflops": world * fl * args.steps / dt / 1e12, "clocks": clocks, "gpu_launches": launches - l0,
            "energies_finite": bool(np.all(np.isfinite(E)))}
    if rank == 0:
        print(json.dumps(line), flush=True)


TTE_VARIANTS = (   # (label, precision, options) of the time-to-E runs
    ("fp64", "fp64", {}),
    ("ozaki", "ozaki", {}),
    ("ozaki6->ozaki", "ozaki", dict(oz_slices=6, refine=True, refine_tol=0.1)),
    ("bf16x3->ozaki", "bf16x3", dict(refine=True, refine_tol=0.1)),
    ("bf16x3", "bf16x3", {}),
    ("tf32x3", "tf32x3", {}),
)


def run_time_to_e(args):
    """Time to a converged energy (Methods: stop when E or ||A|| rises, or |dE| < 1e-6 Eh) on one workload,
    for FP64 FMA, the FP64-accurate Ozaki precision, two precision schedules (Ozaki with 6 slices, or
    BF16x3, until ||A||^2 falls by less than 10 % a step, then Ozaki with 8) and the split precisions:
    one context each, the line search from eps0 (1e-4 for r >= 32, where 1e-3 makes ||A|| rise at the first
    step; else the paper's 1e-3), at most --cap steps; wall time of the host loop (E and ||A||^2 read after
    every step), the stopping energy against FP64's and |E_k - E_k(FP64)| at every iteration.  Then the
    fixed-step leg: --cap steps at eps (1e-4 for r >= 32) in every precision, |E_k - E_k(FP64)| per step."""
    import numpy as np
    import torch
    from paper_2604_02550_gb300 import _lib, api
    p = workload(args.r)
    eps0 = 1e-4 if p.r >= 32 else 1e-3
    eps_fixed = args.eps if args.eps is not None else eps0
    out = {"metric": "time_to_E", "workload": p.name, "r": p.r, "cap": args.cap, "eps0": eps0,
           "stop_rule": "E or ||A|| rises (beyond 1e-12 |E|, 1e-10 ||A||^2), or |dE| < 1e-6 Eh",
           "line_search": {}, "fixed_step": {"eps": eps_fixed}}
    ls = out["line_search"]
    for label, prec, kw in TTE_VARIANTS:
        # a stream of its own: acse_step then replays its CUDA graph (not on the legacy default stream)
        ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, line_search=True, eps0=eps0,
                       stream=torch.cuda.Stream(), **kw)
        with torch.cuda.stream(ctx.stream):
            D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.run_until_stop(D, args.cap)
        dt = time.perf_counter() - t0
        sw, nsw = _lib.acse_schedule_state(ctx.ctx)
        ctx.close()
        ls[label] = {"seconds": dt, "steps": len(res["eps"]), "stop": res["reason"], "accepted": res["accepted"],
                     "E_stop": res["E_stop"], "E": res["E"]}
        if kw.get("refine"):
            ls[label]["switched_after_step"] = nsw if sw else None
    ref = ls["fp64"]
    E_ref = np.array(ref["E"])
    for label, r_ in ls.items():
        m = min(len(r_["E"]), len(E_ref))
        dE = np.abs(np.array(r_["E"][:m]) - E_ref[:m])
        r_["abs_dE_stop_vs_fp64"] = abs(r_["E_stop"] - ref["E_stop"])
        r_["speedup_vs_fp64"] = ref["seconds"] / r_["seconds"]
        r_["abs_dE_per_iteration"] = [float(x) for x in dE]
    for r_ in ls.values():
        del r_["E"]
    fx = out["fixed_step"]
    E64 = None
    for label, prec, kw in (("fp64", "fp64", {}), ("ozaki", "ozaki", {}), ("ozaki6", "ozaki", dict(oz_slices=6)),
                            ("bf16x3", "bf16x3", {}), ("tf32x3", "tf32x3", {})):
        ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, stream=torch.cuda.Stream(), **kw)
        with torch.cuda.stream(ctx.stream):
            D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
            Es = [float(ctx.energy(D))]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.cap):
                E, _, _ = ctx.step(D, eps_fixed)
                Es.append(float(E))
            dt = time.perf_counter() - t0
        ctx.close()
        if E64 is None:
            E64 = np.array(Es)
        dE = np.abs(np.array(Es) - E64)
        fx[label] = {"seconds": dt, "E_final": Es[-1], "max_abs_dE": float(dE.max()),
                     "abs_dE_per_iteration": [float(x) for x in dE]}
    print(json.dumps(out), flush=True)


def run_adjoint_cost(args):
    """Adjoint cost relative to forward on the r = 32 CAS(6e,6o) workload: n Euler steps through acse_step vs
    one acse_residual_backward over the same n steps (every checkpoint given, and only D_0), for the FP64
    FMA path and the Ozaki path (every GEMM of the reverse sweep on the BF16 tensor cores)."""
    import torch
    from paper_2604_02550_gb300 import api
    p = workload(32)
    n, eps = 4, 1e-4
    out = {"metric": "adjoint_cost_ratio", "workload": p.name, "steps": n, "eps": eps,
           "objective": "E(D_n) + 0.5 ||A(D_n)||^2", "runs": {}}

    def timed(fn, reps=3):
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    for prec in ("fp64", "ozaki"):
        ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        ck = [tuple(x.clone() for x in D)]
        for _ in range(n):
            ctx.step(D, eps)
            ck.append(tuple(x.clone() for x in D))
        ctx.backward(ck, n, eps, 1.0, 0.5)                    # warm-up (allocates the adjoint workspace)
        torch.cuda.synchronize()

        def fwd():
            Dw = tuple(x.clone() for x in ck[0])
            for _ in range(n):
                ctx.step(Dw, eps)

        t_f = timed(fwd)
        t_b = timed(lambda: ctx.backward(ck, n, eps, 1.0, 0.5))
        ck_sparse = [ck[0]] + [None] * n                       # only D_0: every D_k recomputed
        t_b0 = timed(lambda: ctx.backward(ck_sparse, n, eps, 1.0, 0.5))
        ctx.close()
        out["runs"][prec] = {"forward_ms": t_f, "backward_ms_all_checkpoints": t_b, "ratio_all_checkpoints": t_b / t_f,
                             "backward_ms_only_D0": t_b0, "ratio_only_D0": t_b0 / t_f}
    out["backward_speedup_ozaki_vs_fp64"] = (out["runs"]["fp64"]["backward_ms_all_checkpoints"] /
                                             out["runs"]["ozaki"]["backward_ms_all_checkpoints"])
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    if args.peaks:
        measure_peaks()
        return
    torch.cuda.set_device(local)
    if args.batch:
        run_batch(args, rank, world)
        return
    if args.time_to_e:
        run_time_to_e(args)
        return
    if args.adjoint:
        run_adjoint_cost(args)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_02550_gb300 import _lib, api
    prec = args.prec or default_prec()
    p = workload(args.r, seed=rank)
    if args.eps is None:
        args.eps = 1e-4 if p.r >= 32 else 1e-3
    stream = torch.cuda.Stream()
    singlet = bool(args.singlet) and prec != "fp64"
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, stream=stream, recon=args.recon, singlet=singlet,
                   gemm_tile=args.gemm_tile)
    with torch.cuda.stream(stream):
        D0 = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        D = tuple(x.clone() for x in D0)
        for _ in range(args.warmup):
            ctx.step(D, args.eps)
    stream.synchronize()
    # clocks: sampled over a window of the same steps (about --sustain-s long, untimed) run directly
    # before the timed region and over the timed region itself, so that a short timed region still
    # has a clock record taken under this load
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t_s = time.perf_counter()
    with torch.cuda.stream(stream):
        while time.perf_counter() - t_s < args.sustain_s:
            for dst, src in zip(D, D0):      # back to D_0 every 100 steps, as the timed region does
                dst.copy_(src)
            for k in range(100):
                ctx.step(D, args.eps)
                if k % 10 == 9:
                    stream.synchronize()
                    if time.perf_counter() - t_s >= args.sustain_s:
                        break
        for dst, src in zip(D, D0):
            dst.copy_(src)
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    def timed_steps():
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                if args.reset_every and k > 0 and k % args.reset_every == 0:
                    for dst, src in zip(D, D0):
                        dst.copy_(src)
                ctx.step(D, args.eps)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    # the timed region: the steps as a user runs them (profiling off, so acse_step replays its CUDA graph);
    # the launch counter is reset here and read after it
    _lib.acse_profile(ctx.ctx, 0)
    ms = timed_steps()
    _, _, launches = _lib.acse_profile_read(ctx.ctx)
    # the GEMM's launch duration: CUDA events on the context's stream around every GEMM launch, over the
    # same K steps run once more directly (the events would split the step's graph, so the headline
    # region above runs without them)
    for dst, src in zip(D, D0):
        dst.copy_(src)
    _lib.acse_profile(ctx.ctx, 1)
    ms_profiled = timed_steps()
    gemm_ms, gemm_n, _ = _lib.acse_profile_read(ctx.ctx)
    _lib.acse_profile(ctx.ctx, 0)
    clocks = sampler.stop()
    ms_max = max_over_ranks(ms, dist)
    per_step = ms_max / args.steps
    value = whole_job_rate(EVALS_PER_STEP * args.steps, world, ms_max)
    fl_alg = flops_per_pass(p.r)                       # 32 r^6: the unpacked formulation
    # what the GEMM launch executes (the same-spin pair GEMMs on packed pairs on every path but FP64 FMA)
    fl = fl_alg if prec == "fp64" else flops_per_pass(p.r, packed=True, singlet=singlet)
    split = 3 if prec in ("bf16x3", "tf32x3") else 1
    if prec == "ozaki":
        split = oz_moduli_count(OZ_SLICES, 2 * p.r * p.r)   # bf16 residue products per FP64 GEMM
    # dominant kernel: the grouped O(r^6) GEMM launch (one per contraction pass)
    gemm_avg_s = gemm_ms / max(gemm_n, 1) / 1e3
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        peaks = json.load(open(PEAKS_FILE))
    if prec == "fp64":
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                "peak_source": "measured cuBLAS DGEMM 8192^3 on this pool (bench.py --peaks); DFMA pipe"}
        ach = fl / gemm_avg_s / 1e12
    elif prec in ("bf16x3", "ozaki"):
        measured = "bf16_tflops" in peaks
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": peaks["bf16_tflops"] if measured else 1900.0,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" if measured else "fallback 1.9 PFLOP/s"}
        ach = split * fl / gemm_avg_s / 1e12
    else:
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": TF32_PEAK_TFLOPS,
                "peak_source": "measured cuBLAS TF32 8192^3 on this pool (bench.py --peaks)"}
        ach = split * fl / gemm_avg_s / 1e12
    roof.update({"achieved": ach, "frac": ach / roof["peak"], "traffic": gemm_traffic(prec) if p.r == 48 else None,
                 "kernel": "grouped O(r^6) GEMM",
                 "flops_per_launch": split * fl,
                 "flops_note": {"fp64": "2MNK, 32 r^6 per pass",
                                "ozaki": f"bf16 residue products of the modular Ozaki scheme: {split} per FP64 "
                                         f"GEMM ({OZ_SLICES} slices: {min(6 * OZ_SLICES, 53)}-bit integer rows, "
                                         f"{split} moduli), 2MNK each, same-spin pair GEMMs on pairs i<j; the "
                                         f"timed launch includes the reconstruction kernel"}.get(
                     prec, "2MNK of the GEMMs the launch executes (same-spin pair GEMMs on pairs i<j)"),
                 "launch_ms": 1e3 * gemm_avg_s,
                 "launch_timing": "CUDA events around each GEMM launch on the context's stream, over a second run "
                                  "of the same steps issued directly (events would split the step's CUDA graph); "
                                  f"that run took {ms_profiled / args.steps:.4f} ms a step",
                 "gemm_share_of_step": 2 * 1e3 * gemm_avg_s / per_step,
                 "timed_launches": gemm_n})
    clocks["window"] = (f"sampled every 100 ms over {args.sustain_s:.1f} s of the same untimed steps directly before "
                        f"the timed region and over the timed region")
    line = {"metric": "acse_residual_evals_per_s", "value": value, "unit": "residual evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True,
            "evals_per_step": EVALS_PER_STEP, "acse_steps_per_s": value / EVALS_PER_STEP,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "ozaki": "f64 (Ozaki: bf16 residues, exact f32 chunk sums, CRT to f64)"}.get(
                prec, f"{prec} (f32 accumulate)"),
            "data": "synthetic",
            "config": {"workload": p.name, "r": p.r, "N": p.N, "prec": prec, "recon": args.recon, "eps": args.eps,
                       "singlet": singlet,
                       "step": "acse_step: residual + update + axpy + energy (two residual evaluations)",
                       "reset_every": args.reset_every,
                       "l2": "inputs larger than L2 (about 1.5 GB of r^4 tensors touched per step)",
                       "parallelism": f"replicas x{world}"},
            "tflops": world * 2 * fl / (ms_max / 1e3 / args.steps) / 1e12,
            "tflops_32r6": world * 2 * fl_alg / (ms_max / 1e3 / args.steps) / 1e12,
            "gpu_launches": launches, "clocks": clocks, "roofline": roof}
    ctx_e2e = None
    if not args.no_e2e and rank == 0:
        # end to end: host (pinned) buffers through the same C ABI; H2D, compute, D2H inside the loop
        Dh = [torch.from_numpy(x.copy()).pin_memory() for x in (p.Daa, p.Dab, p.Dbb)]
        Eh = torch.zeros(1, dtype=torch.float64).pin_memory()
        Nh = torch.zeros(1, dtype=torch.float64).pin_memory()
        Sh = torch.zeros(1, dtype=torch.float64).pin_memory()
        ctx_e2e = ctx
        for _ in range(2):
            _lib.acse_step(ctx.ctx, *Dh, args.eps, Eh, Nh, Sh)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _lib.acse_step(ctx.ctx, *Dh, args.eps, Eh, Nh, Sh)
        dt = time.perf_counter() - t0
        n4 = p.r ** 4
        line["e2e"] = {"value": EVALS_PER_STEP * args.steps / dt, "unit": "residual evals/s",
                       "h2d_bytes_per_step": 3 * n4 * 8,
                       "d2h_bytes_per_step": 3 * n4 * 8 + 3 * 8,
                       "how": "acse_step on pinned host D blocks: staged H2D, step, D2H of D, E, ||A||^2, eps"}
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        v, dt, cores = cpu_oracle_timing(p, 1)
        line["cpu_baseline"] = {"value": v, "unit": "residual evals/s", "cores": cores, "kind": "oracle",
                                "sample": f"one FP64 oracle residual evaluation of {p.name} ({dt:.1f} s)"}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
