"""Benchmark: Kohn-Sham density-matrix solves per second, (H, S) -> (P, W), on one GB300.

Workload: the 3D-cluster synthetic problem of n = 16384 basis functions (1093 atoms x 15
functions, N_el = 4096, n_state = 2048, integer occupation, lambda_min(S) rescaled to
>= 1e-2), inputs device-resident. One step = elsi_dm_real + elsi_get_edm_real through
the C ABI, including the Cholesky of S (no reuse of the factor between steps). The
FP32-reduction + refinement route is the measured arm; the binary64 route is timed
beside it and both results are compared (relative Frobenius error of P).

`--impl reference` times the FP64 CPU oracle instead (the paper has no runnable
reference); under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("KS solves/s (H,S→P,W) at n=16384: FP32+refine vs FP64 GPU, rel err ≤1e-9")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
L2_BYTES = 129 * 2 ** 20  # L2 of the GB300
# binary64 FMA rate of the chip, derived from unit counts: 152 SMs x 2 DFMA/clk/SM x 2 flop
FP64_FLOP_PER_CLK = 152 * 2 * 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the binary64 comparison arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the several-problem workloads (k-point batch, mixed sizes)")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--fd-check", type=int, default=0, metavar="N",
                    help="instead of the benchmark: the free-energy derivative check at size N "
                         "(binary32 + refinement forward, Fermi-Dirac kT = 0.01, dF/dH = P and "
                         "dF/dS = -W against central differences on random symmetric directions)")
    ap.add_argument("--fd-dirs", type=int, default=32)
    ap.add_argument("--lambda-min", type=float, default=None,
                    help="force lambda_min(S) to this value (the overlap-conditioning sweep)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n: int, tau: float | None = None):
    import ksinputs
    if n == 16384:
        p = ksinputs.workload("cluster3d-n16384", tau=tau)
    elif n == 8192:
        p = ksinputs.workload("cluster3d-n8192", tau=tau)
    else:
        p = ksinputs.cluster_problem(n, seed=2, tau=1e-2 if tau is None else tau,
                                     force_tau=tau is not None)
    return p


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax or None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n_target: int, sample_n: int = 1024):
    """Times the FP64 CPU oracle on a bounded sample (the same 3D-cluster construction at
    sample_n) and scales its solve time by (n_target / sample_n)^3 to solves/s at n_target
    (optimistic for the oracle: its Jacobi sweep count also grows with n)."""
    import ksinputs
    import oracle
    oracle.build()
    p = ksinputs.cluster_problem(sample_n, seed=2)
    t0 = time.perf_counter()
    oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    dt = time.perf_counter() - t0
    scaled = dt * (n_target / sample_n) ** 3
    return {"value": 1.0 / scaled, "unit": "solves/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"one full oracle solve at n={sample_n} (same 3D-cluster construction) "
                      f"took {dt:.2f} s; scaled by (n/{sample_n})^3 to n={n_target}"}


def workload_config(n: int, world: int, tau: float | None = None) -> dict:
    """The config object both arms print: the workload by what it is, with its sizes (the
    arithmetic of each arm is in its own "dtype" and "route" keys, not in the config)."""
    import ksinputs
    c = ksinputs.WORKLOADS.get(f"cluster3d-n{n}")
    nel = int(c["n_electron"]) if c else n // 4
    k = int(c["n_state"]) if c else max(1, -(-nel // 2))
    gb = n * n * 8 / 1e9
    l2 = ("inputs (2 x %.2g GB) larger than L2; no flush" % gb) if 2 * n * n * 8 > L2_BYTES else \
        ("inputs (2 x %.2g GB) within L2" % gb)
    lam = "lambda_min(S) >= 1e-2" if tau is None else f"lambda_min(S) = {tau:g}"
    return {"workload": f"3D-cluster KS problem n={n}, N_el={nel}, n_state={k}, integer "
                        f"occupation, {lam}",
            "parallelism": f"replicas x{world}", "l2": l2}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        cpu_baseline(args.n)
    for _ in range(args.steps):
        steps.append(cpu_baseline(args.n))
    val = sum(s["value"] for s in steps) / len(steps)
    cb = dict(steps[-1])
    cb["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / val, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n, world, args.lambda_min),
            "route": "binary64 CPU oracle (Cholesky + cyclic Jacobi)",
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def algorithmic_flops(n: int, k: int) -> float:
    # Cholesky n^3/3, standard form ~n^3 (symmetric), full->band 4n^3/3, back-transforms
    # through Q2, Q1 and L^-T for k vectors 5 n^2 k, P and W 2 n^2 k (8/3 n^3 + 7 n^2 k)
    return 8.0 / 3.0 * n ** 3 + 7.0 * n * n * k


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    import paper_1705_11191_gb300 as egb

    torch.cuda.set_device(local)
    if args.fd_check:
        if rank == 0:
            print(json.dumps(fd_check(egb, torch, args.fd_check, args.fd_dirs)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = egb.PREC_FP32_REFINE if args.precision == "fp32_refine" else egb.PREC_FP64
    p = workload(args.n, args.lambda_min)
    n, k = p.n, p.n_state
    dev = torch.device("cuda", local)
    H = torch.from_numpy(np.ascontiguousarray(p.h)).to(dev)
    S = torch.from_numpy(np.ascontiguousarray(p.s)).to(dev)
    P = torch.empty((n, n), dtype=torch.float64, device=dev)
    W = torch.empty((n, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make_handle(pr):
        hd = egb.Handle(n, k, p.n_electron)
        hd.set_stream(stream)
        hd.set_precision(pr)
        return hd

    hd = make_handle(prec)

    def step():
        _, e = hd.dm_real(H, S, out=P)
        hd.get_edm(out=W)
        return e

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stage_acc = {}
    launches0 = egb.launch_count()
    with ClockSampler(local) as cs:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            energy = step()
            for kk, v in hd.stage_times().items():
                stage_acc[kk] = stage_acc.get(kk, 0.0) + v
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (egb.launch_count() - launches0) // args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    stages = {kk: v / args.steps for kk, v in stage_acc.items()}
    iters, orth = hd.refine_info()
    value = world * 1000.0 / ms

    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if prec == egb.PREC_FP32_REFINE else "f64", "data": "synthetic",
           "config": workload_config(n, world, args.lambda_min),
           "route": args.precision,
           "lambda_min_s": p.lambda_min_s,
           "stages_ms": {kk: round(v, 3) for kk, v in stages.items()},
           "refine_iters": iters, "refine_fell_back_to_fp64": iters == -1, "orth_err": orth,
           "tflops_algorithmic": algorithmic_flops(n, k) / (ms * 1e-3) / 1e12,
           "clocks": cs.summary()}

    # roofline of the dominant kernel: in the binary32 route the largest single kernel is
    # the Q2 back-transformation (one launch per solve; the full-to-band stage is longer but
    # is hundreds of panel-factorisation and GEMM launches); else the largest stage
    dom = "back_q2" if prec == egb.PREC_FP32_REFINE else max(stages, key=stages.get)
    out["roofline"] = roofline_for(dom, stages[dom], n, k, prec, out["clocks"],
                                   refine_iters=max(iters, 0))
    out["stages_roofline"] = {st: roofline_for(st, v, n, k, prec, out["clocks"],
                                               refine_iters=max(iters, 0))
                              for st, v in stages.items() if v > 0.0}

    # binary64 arm and the relative error of P between the two routes
    if not args.no_fp64 and rank == 0 and prec == egb.PREC_FP32_REFINE:
        h64 = make_handle(egb.PREC_FP64)
        P64 = torch.empty_like(P)
        h64.dm_real(H, S, out=P64)  # warm-up
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        _, e64 = h64.dm_real(H, S, out=P64)
        W64 = h64.get_edm()
        t1.record(stream)
        torch.cuda.synchronize()
        ms64 = t0.elapsed_time(t1)
        ev32 = hd.get_eval()
        ev64 = h64.get_eval()
        out["max_abs_err_eval_vs_fp64"] = float((ev32 - ev64).abs().max())
        relp = float(torch.linalg.norm(P - P64) / torch.linalg.norm(P64))
        relw = float(torch.linalg.norm(W - W64) / torch.linalg.norm(W64))
        out["fp64_gpu"] = {"value": 1000.0 / ms64, "unit": "solves/s", "ms_per_step": ms64,
                           "stages_ms": {kk: round(v, 3) for kk, v in h64.stage_times().items()}}
        out["rel_err_P_vs_fp64"] = relp
        out["rel_err_W_vs_fp64"] = relw
        out["abs_err_energy_vs_fp64"] = abs(energy - e64)
        out["speedup_vs_fp64_gpu"] = ms64 / ms
        h64.close()
        del P64, W64

    # end to end through the host-buffer entry point (pinned buffers)
    if not args.no_e2e:
        hh = torch.from_numpy(np.ascontiguousarray(p.h)).pin_memory()
        sh = torch.from_numpy(np.ascontiguousarray(p.s)).pin_memory()
        ph = torch.empty((n, n), dtype=torch.float64).pin_memory()
        wh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        hd.dm_real_host(hh, sh, ph, wh)
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            hd.dm_real_host(hh, sh, ph, wh)
        dt = (time.perf_counter() - t0) / e2e_steps
        out["e2e"] = {"value": world / dt, "unit": "solves/s",
                      "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": 2 * n * n * 8,
                      "steps": e2e_steps}

    if not args.no_batch and rank == 0:
        out["batch_workloads"] = batch_workloads(egb, torch, dev, stream, args.batch_steps)

    out["gpu_launches"] = launches
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(n)
    if rank == 0:
        print(json.dumps(out), flush=True)
    hd.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def fd_check(egb, torch, n: int, ndirs: int, h: float = 1e-6, kt: float = 0.01) -> dict:
    """Derivatives of the Mermin free energy F = E_band - kT S_ent of the 3D-cluster problem
    of size n (seed 5, N_el = n/4), binary32 + refinement forward, Fermi-Dirac kT = 0.01 Ha,
    mu bisected to |N(mu) - N_el| <= 1e-12, n_state = N_el/2 + n/8 (the occupation of the
    last computed state is reported). The backward gives dF/dH = P and dF/dS = -W
    (elsi_dm_adjoint_real through KSFreeEnergy). Each of ndirs random symmetric directions
    D (entries (X + X^T)/2 with X_ij ~ N(0,1), generator seed 6) is checked by central
    differences, (F(H + hD) - F(H - hD)) / 2h against <dF/dH, D>, and likewise for S.
    Memory: H, S, the two gradients, D and one density-matrix buffer on the caller's side
    (6 n^2 binary64 values; H and S are perturbed in place and restored)."""
    import ksinputs
    from paper_1705_11191_gb300 import autograd as ega
    dev = torch.device("cuda")
    t0 = time.perf_counter()
    H, S, nel, _, lam = ksinputs.cluster_problem_torch(n, 5, dev)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    nstate = min(n, int(nel // 2 + n // 8))
    gen_s = time.perf_counter() - t0
    hd = egb.Handle(n, nstate, nel)
    hd.use_current_stream()
    hd.set_precision(egb.PREC_FP32_REFINE)
    hd.set_broadening(egb.OCC_FERMI, kt)
    hd.set_occ_accuracy(1e-12)
    H.requires_grad_(True)
    S.requires_grad_(True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    F = ega.free_energy(H, S, hd)
    torch.cuda.synchronize()
    fwd_s = time.perf_counter() - t1
    iters, orth = hd.refine_info()
    occ_last = float(hd.get_occ()[-1])
    t2 = time.perf_counter()
    F.backward()
    torch.cuda.synchronize()
    bwd_s = time.perf_counter() - t2
    F0 = float(F)
    del F
    gH, gS = H.grad, S.grad
    H.requires_grad_(False)
    S.requires_grad_(False)
    H.grad = None
    S.grad = None
    torch.cuda.empty_cache()
    Pbuf = torch.empty((n, n), dtype=torch.float64, device=dev)
    gen = torch.Generator(device=dev).manual_seed(6)
    rows = []

    def energy():
        _, e = hd.dm_real(H, S, out=Pbuf)
        return e + hd.get_entropy()

    with torch.no_grad():
        for q in range(ndirs):
            D = torch.randn((n, n), dtype=torch.float64, device=dev, generator=gen)
            D.add_(D.T.contiguous()).mul_(0.5)
            torch.cuda.empty_cache()
            for which, X, g in (("H", H, gH), ("S", S, gS)):
                an = float((g * D).sum())
                X.add_(D, alpha=h)
                fp = energy()
                X.add_(D, alpha=-2.0 * h)
                fm = energy()
                X.add_(D, alpha=h)
                fd = (fp - fm) / (2.0 * h)
                rows.append({"dir": q, "wrt": which, "analytic": an, "central_difference": fd,
                             "abs_err": abs(fd - an), "rel_err": abs(fd - an) / max(abs(an), 1e-300)})
            del D
    hd.close()
    errs = [r["rel_err"] for r in rows]
    rms = (sum(r["analytic"] ** 2 for r in rows) / max(1, len(rows))) ** 0.5
    return {"check": "free-energy derivatives by central differences", "n": n,
            "n_electron": nel, "n_state": nstate, "kT": kt, "lambda_min_s": lam,
            "occ_of_last_state": occ_last, "F": F0, "refine_iters": iters,
            "orth_err": orth, "forward_s": fwd_s, "backward_s": bwd_s,
            "input_generation_s": gen_s, "step": h, "directions": ndirs,
            "max_rel_err": max(errs) if errs else None,
            "median_rel_err": sorted(errs)[len(errs) // 2] if errs else None,
            "max_abs_err": max(r["abs_err"] for r in rows) if rows else None,
            "rms_analytic": rms, "rows": rows}


def _bucket(n: int) -> int:
    q = 0
    while (1 << q) < n:
        q += 1
    return 1 << q


def batch_workloads(egb, torch, dev, stream, steps: int) -> dict:
    """The several-problem path (k-points and spin channels, SINGLE_PROC mode) on its two
    synthetic batches, binary32 + refinement, autotuned reduction and concurrency:
      kpoints-64x2048: 64 complex Hermitian k-point problems of n = 2048 (Gamma-centred
        4x4x4 grid, 27 real lattice blocks, seed 3), Fermi-Dirac kT = 0.01 Ha, one
        chemical potential over all k-points (weights 1/64, N_el = 512 per cell),
        n_state = 640;
      mixed-200: 200 real problems, n log-uniform over 256..4096 (sizes seed 4, problem i
        seed 1000 + i), integer occupation with N_el = n/4 each.
    One warm-up batch (the autotuner runs on first use), then `steps` timed batches (CUDA
    events on the solve stream; the mixed batch is timed per size bucket, one batched
    call per bucket). Parity: one problem per batch / bucket solved alone in the binary32
    route and in the binary64 route, relative Frobenius error of P between the two."""
    import ksinputs
    out = {}

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- k-point batch
    t0 = time.perf_counter()
    n, nk, kt = 2048, 64, 0.01
    kset = ksinputs.kpoint_set(n, grid=4, seed=3, device=dev)
    nel = float(n // 4)
    nstate = 640
    hams = [h.transpose(0, 1).contiguous() for (_, h, _, _) in kset]
    ovls = [s_.transpose(0, 1).contiguous() for (_, _, s_, _) in kset]
    del kset
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    hd = egb.Handle(n, nstate, nel)
    hd.set_stream(stream)
    hd.set_precision(egb.PREC_FP32_REFINE)
    hd.set_broadening(egb.OCC_FERMI, kt)
    hd.set_occ_accuracy(1e-12)
    wts = [1.0 / nk] * nk
    t1 = time.perf_counter()
    hd.dm_batched(hams, ovls, [nstate] * nk, nel, weights=wts, shared_mu=True, inputs_colmajor=True)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t1
    a, b_ = ev_pair()
    a.record(stream)
    for _ in range(steps):
        P, W, E, mu = hd.dm_batched(hams, ovls, [nstate] * nk, nel, weights=wts, shared_mu=True,
                                    inputs_colmajor=True)
    b_.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b_) / steps
    tune = hd.batch_tuning(n, True)
    del P, W
    hd.close()
    # parity of k-point 0 alone: binary32 route vs binary64 route (own chemical potential)
    h0 = hams[0].transpose(0, 1).contiguous()
    s0 = ovls[0].transpose(0, 1).contiguous()
    res = {}
    for pr in (egb.PREC_FP32_REFINE, egb.PREC_FP64):
        with egb.Handle(n, nstate, nel) as h1:
            h1.set_stream(stream)
            h1.set_precision(pr)
            h1.set_broadening(egb.OCC_FERMI, kt)
            h1.set_occ_accuracy(1e-12)
            p1, e1 = h1.dm_complex(h0, s0)
            res[pr] = (p1, e1)
    relp = float(torch.linalg.norm(res[1][0] - res[0][0]) / torch.linalg.norm(res[0][0]))
    out["kpoints-64x2048"] = {
        "problems": nk, "n": n, "complex": True, "n_state": nstate, "kT": kt,
        "problems_per_s": nk / (ms * 1e-3), "ms_per_batch": ms, "steps": steps,
        "mu": mu, "first_call_s_including_autotune": first_s, "input_generation_s": gen_s,
        "tuning": None if tune is None else dict(zip(("band_width", "elpa_solver", "streams"), tune)),
        "parity_kpoint0_rel_err_P_vs_fp64": relp,
        "parity_kpoint0_abs_err_energy_vs_fp64": abs(res[1][1] - res[0][1])}
    del hams, ovls, res, h0, s0
    torch.cuda.empty_cache()

    # ---- mixed sizes
    t0 = time.perf_counter()
    sizes = ksinputs.mixed_sizes(200, seed=4)
    probs = [ksinputs.cluster_problem_torch(nn, 1000 + i, dev) for i, nn in enumerate(sizes)]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    groups = {}
    for i, nn in enumerate(sizes):
        groups.setdefault(_bucket(nn), []).append(i)
    hd = egb.Handle(4096, 1024, 2048.0)
    hd.set_stream(stream)
    hd.set_precision(egb.PREC_FP32_REFINE)

    def run_bucket(idx):
        return hd.dm_batched([probs[i][0] for i in idx], [probs[i][1] for i in idx],
                             [probs[i][3] for i in idx], [probs[i][2] for i in idx],
                             shared_mu=False)

    t1 = time.perf_counter()
    for bk in sorted(groups):
        run_bucket(groups[bk])
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t1
    per = {}
    total_ms = 0.0
    for bk in sorted(groups):
        idx = groups[bk]
        a, b_ = ev_pair()
        a.record(stream)
        for _ in range(steps):
            P, W, E, mus = run_bucket(idx)
        b_.record(stream)
        torch.cuda.synchronize()
        bms = a.elapsed_time(b_) / steps
        total_ms += bms
        i0 = idx[0]
        with egb.Handle(sizes[i0], probs[i0][3], probs[i0][2]) as h64:
            h64.set_stream(stream)
            h64.set_precision(egb.PREC_FP64)
            p64, _ = h64.dm_real(probs[i0][0].clone(), probs[i0][1])
        relp = float(torch.linalg.norm(P[0] - p64) / torch.linalg.norm(p64))
        tune = hd.batch_tuning(bk, False)
        per[f"n<={bk}"] = {
            "problems": len(idx), "ms_per_batch": bms, "solves_per_s": len(idx) / (bms * 1e-3),
            "tuning": None if tune is None else dict(zip(("band_width", "elpa_solver", "streams"), tune)),
            "parity_rel_err_P_vs_fp64": relp, "parity_problem_n": sizes[i0]}
        del P, W
    hd.close()
    out["mixed-200"] = {"problems": len(sizes), "problems_per_s": len(sizes) / (total_ms * 1e-3),
                        "ms_per_batch_sum_of_buckets": total_ms, "steps": steps,
                        "first_calls_s_including_autotune": first_s, "input_generation_s": gen_s,
                        "buckets": per}
    del probs
    torch.cuda.empty_cache()
    return out


# dominant kernel of each stage of the binary32+refinement route (one launch per solve
# unless noted) and the arithmetic it runs on
_STAGE_KERNEL = {
    "cholesky": ("potrf_diag_kernel + gemm_tf32x3_kernel", "tf32"),
    "standard_form": ("gemm_tf32x3_kernel (blocked triangular solves)", "tf32"),
    "full_to_band": ("panel_qr_kernel + w_stage kernels + gemm_tf32x3_kernel", "tf32"),
    "band_to_tri": ("chase_kernel", None),
    "tridiag_solve": ("bisect_kernel + twisted_kernel", None),
    "back_q2": ("q2_apply_tc5_kernel (two launches: block ranges) + q2_factor_kernel", "tf32"),
    "back_q1": ("gemm_tf32x3_kernel", "tf32"),
    "back_subst": ("gemm_tf32x3_kernel (blocked triangular solve)", "tf32"),
    "refine": ("ozaki_gemm_tc_kernel (all launches of the stage)", "bf16"),
    "occupation": ("occupation_kernel", None),
    "density": ("ozaki_gemm_tc_kernel (P and W)", "bf16"),
}
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tf32 / bf16 tensor rates

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a stage's kernels from one
# ncu capture, valid while the kernel's source file is unchanged (sha256 prefix). The Q2
# capture is at n = 8192 (the n = 16384 workspace is too large for a multi-pass capture);
# its traffic is one read and one write of the remaining rows of Z per block of 64 sweeps,
# which grows as n^3 once Z exceeds L2 (as it does at 8192 and 16384), so it is scaled by
# (n / 8192)^3.
MEASURED_TRAFFIC = {
    "back_q2": {"kernel": "q2_apply_tc5_kernel", "source": "paper_1705_11191_gb300/csrc/q2tc.cu",
                "sha256_16": "a7bd6373b70be307", "n": 8192, "bytes": 15318903552 + 16249897472},
}


def stage_traffic(stage: str, n: int):
    """Traffic per solve of the stage's kernels at size n, or None when no capture matches."""
    import hashlib
    m = MEASURED_TRAFFIC.get(stage)
    if not m or n < m["n"]:
        return None
    try:
        with open(os.path.join(ROOT, m["source"]), "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != m["sha256_16"]:
        return None  # the kernel changed since the counters were taken
    return m["bytes"] * (n / m["n"]) ** 3
OZAKI_PRODUCTS = 28  # bf16 digit products per binary64-accurate product (7 digits, 8 levels)


def _peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "of measured"
    except OSError:
        return {}, "of fallback"


def stage_work(stage: str, n: int, k: int, prec: int, refine_iters: int = 4, band: int = 64):
    """Algorithmic work of one stage per solve: (amount, unit). Flops follow the count of
    the hot-path table ((8/3) n^3 + 7 n^2 k in total): Cholesky n^3/3, standard form n^3
    (the symmetric two-sided solve), full->band 4n^3/3, back-transformations 2n^2 N each and
    back-substitution n^2 N for the N vectors carried (N = n in the binary32 route, which
    back-transforms all vectors for the refinement; k in the binary64 route), P and W n^2 k
    each (symmetric products). The refinement counts its binary64-accurate products per pass
    (H X, S X: 2n^2 k each; X^T Y_H, X^T Y_S: 2n k^2 each), passes = iterations + the final
    Rayleigh-Ritz. The bulge chase is counted in bytes of band traffic: per (sweep, step)
    task the b x b blocks X and D are read and written."""
    nv = n if prec == 1 else k
    if stage == "band_to_tri":
        tasks = sum((n - 2 - j) // band + 1 for j in range(n - 2))
        return tasks * 4.0 * band * band * (4 if prec == 1 else 8), "bytes"
    flops = {
        "cholesky": n ** 3 / 3.0,
        "standard_form": 1.0 * n ** 3,
        "full_to_band": 4.0 * n ** 3 / 3.0,
        "back_q2": 2.0 * n * n * nv,
        "back_q1": 2.0 * n * n * nv,
        "back_subst": 1.0 * n * n * nv,
        "density": 2.0 * n * n * k,
        "refine": (4.0 * n * n * k + 4.0 * k * k * n) * (refine_iters + 1),
    }.get(stage)
    return flops, "flops"


def roofline_for(stage: str, stage_ms: float, n: int, k: int, prec: int, clocks: dict,
                 refine_iters: int = 4, band: int = 64):
    """Roofline entry of one stage: its algorithmic work per solve (stage_work) divided by
    the stage's device time (CUDA events recorded on the solve stream around the stage).
    Tensor-core stages take the measured sustained bf16 rate of MEASURED_PEAKS.json (times
    the nominal tf32/bf16 ratio for tf32 work; binary64-accurate Ozaki products are
    counted as their 28 bf16 digit products); the bulge chase takes band bytes against the
    measured copy bandwidth; binary64 (SIMT) and ALU-bound stages take the binary64 FMA
    rate derived from unit counts (152 SMs x 2 DFMA/clk x 2070 MHz)."""
    peaks, src = _peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    hbm = peaks.get("hbm_gbs") or 6800.0
    kern, dt = _STAGE_KERNEL.get(stage, (stage, None))
    if prec == 0:
        dt = None
    out = {"stage": stage, "kernel": kern, "ms": round(stage_ms, 3),
           "traffic": stage_traffic(stage, n) if prec == 1 else None}
    sec = stage_ms * 1e-3
    work, unit = stage_work(stage, n, k, prec, refine_iters, band)
    if unit == "bytes":
        ach = work / sec / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                   peak_note=f"hbm_gbs {src} (copy bandwidth); band bytes = tasks x 4 b^2 x elem")
        return out
    if work is None or dt is None:
        fp64_peak = FP64_FLOP_PER_CLK * 2070e6 / 1e12
        ach = work / sec / 1e12 if work else None
        out.update(bound="alu", achieved=ach, peak=fp64_peak, unit="TFLOP/s",
                   frac=(ach / fp64_peak) if ach else None,
                   peak_note="binary64 FMA rate derived from 152 SMs x 2 DFMA/clk x 2070 MHz" +
                             ("" if work else "; no dense-flop count for this stage"))
        return out
    if dt == "bf16":
        tc_work = OZAKI_PRODUCTS * work
        peak = bf16
        note = (f"bf16_tflops_sustained {src}; {OZAKI_PRODUCTS} bf16 digit products per "
                "binary64-accurate flop")
    else:
        tc_work = work
        peak = bf16 * TF32_PER_BF16
        note = (f"bf16_tflops_sustained {src} x nominal tf32/bf16 ratio 1.1/2.25; tf32 work "
                "counted once (the three split products are not counted)")
    ach = tc_work / sec / 1e12
    out.update(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
               algorithmic_tflops=work / sec / 1e12, peak_note=note)
    return out


if __name__ == "__main__":
    main()
