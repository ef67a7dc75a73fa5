"""Benchmark of the ETD2RK-DS step on GB300.

Default workload (N = 1): 2D FitzHugh-Nagumo, n = 4096 interior points per axis,
two fields, kappa_u = 1e-3, kappa_v = 5e-3, eps = 0.01, a = 0.5, b = 0.1,
tau = 1e-2, Pade P_{0,2}, seeded U[-0.1, 0.1] fields, in the FP64-split
precision: FP64 fields and state, every product with P as exact products of
balanced 8-bit integer slices on the BF16 tensor cores. It is the precision that stays
within 1e-6 of the FP64 oracle over this configuration's whole run of 1000 steps
(9.5e-11 measured); split BF16 x6 (--precision bf16x6) is about six times faster
and within 1e-6 for the first 100 steps, 4.6e-6 over the 1000.
A "step" is one ETD2RK-DS time step (eq. (13)-(14)): two reaction kernels and
eight transform passes over both fields.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--precision P]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
    python bench.py --accuracy --workload NAME [--precisions P1,P2]
        # error vs the FP64 oracle over the configuration's whole run length,
        # beside the floors of FP32 input rounding and of the oracle's FP32 shadow

Prints one JSON line (rank 0). With N > 1 (torchrun), every rank advances its
own replica of the workload (the problem has no data-parallel exchange; see
the design notes): value = all ranks' unknown-updates / max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FHN = (1.0, 0.01, 0.5, 0.1)  # c3, eps, a, b

WORKLOADS = {
    # name: (d, n, kappa_u, kappa_v or None, q, tau, reaction, description)
    "fhn2d_4096": (2, 4096, 1e-3, 5e-3, 0.0, 1e-2, "fhn",
                   "2D FitzHugh-Nagumo n=4096 (2 fields), kappa_u=1e-3 kappa_v=5e-3 eps=0.01 a=0.5 b=0.1 tau=1e-2"),
    "fhn2d_2048": (2, 2048, 1e-3, 5e-3, 0.0, 1e-2, "fhn",
                   "2D FitzHugh-Nagumo n=2048 (2 fields), kappa_u=1e-3 kappa_v=5e-3 eps=0.01 a=0.5 b=0.1 tau=1e-2"),
    "ac3d_256": (3, 256, 1e-3, None, 0.1, 5e-3, "allen_cahn", "3D Allen-Cahn n=256, kappa=1e-3 q=0.1 tau=5e-3"),
    # grids with n + 1 a power of two, for the fast sine transform comparison (--precision dst32)
    "fhn2d_4095": (2, 4095, 1e-3, 5e-3, 0.0, 1e-2, "fhn",
                   "2D FitzHugh-Nagumo n=4095 (2 fields), kappa_u=1e-3 kappa_v=5e-3 eps=0.01 a=0.5 b=0.1 tau=1e-2"),
    "ac3d_255": (3, 255, 1e-3, None, 0.1, 5e-3, "allen_cahn", "3D Allen-Cahn n=255, kappa=1e-3 q=0.1 tau=5e-3"),
    "ac3d_384": (3, 384, 1e-3, None, 0.1, 5e-3, "allen_cahn", "3D Allen-Cahn n=384, kappa=1e-3 q=0.1 tau=5e-3"),
    "ac2d_64": (2, 64, 1e-2, None, 0.0, 1e-3, "allen_cahn", "2D Allen-Cahn n=64, kappa=1e-2 q=0 tau=1e-3"),
    "adjoint3d_128": (3, 128, 1e-3, 5e-3, 0.0, 1e-2, "fhn",
                      "gradient of ||u(T) - u_target||^2 over 400 steps of 3D FitzHugh-Nagumo n=128 (2 fields), "
                      "kappa_u=1e-3 kappa_v=5e-3 eps=0.01 a=0.5 b=0.1 tau=1e-2, checkpoints every 20 steps; "
                      "u_target from the same run at kappa_u (1 + 1e-2)"),
    "ensemble512": (2, None, None, 5e-3, 0.0, None, "fhn",
                    "512 independent 2D FitzHugh-Nagumo instances, n uniform on {64,96,...,512}, kappa_u log-uniform "
                    "[1e-4,1e-2], tau uniform [1e-3,1e-2], kappa_v=5e-3 eps=0.01 a=0.5 b=0.1"),
}
# run length of each workload's configuration (the accuracy check runs all of it)
RUN_STEPS = {"fhn2d_4096": 1000, "fhn2d_2048": 1000, "fhn2d_4095": 1000, "ac3d_256": 200, "ac3d_384": 200,
             "ac3d_255": 200, "ac2d_64": 100, "ensemble512": 500, "adjoint3d_128": 400}
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates
F64_PRECISIONS = ("fp64", "fp64split", "fp64split40", "fp64split32")  # precisions with FP64 fields
# the arithmetic each precision computes in
DTYPE = {"fp64": "f64", "fp32": "f32", "tf32": "tf32 (f32 fields)",
         "tf32x3": "tf32x3 (f32 fields, double-float spectral state)",
         "tf32x6": "tf32x6 (f32 fields, double-float spectral state)",
         "bf16x3": "bf16x3 (f32 fields, double-float spectral state)",
         "bf16x6": "bf16x6 (f32 fields, double-float spectral state)",
         "fp64split": "f64 (f64 fields and state; products as 21 exact bf16 slice products)",
         "fp64split40": "f64 (f64 fields and state; products as 15 exact bf16 slice products, 40-bit operands)",
         "fp64split32": "f64 (f64 fields and state; products as 10 exact bf16 slice products, 32-bit operands)",
         "dst32": "f32 (fast sine transforms)"}
# DRAM traffic records (ncu, per launch of the per-step pass) of the default
# workload, with the kernel sources they are valid for
TRAFFIC_RECORDS = {
    "bf16x6": ("profiles/gemm_tc_accurate_bf16x6_fhn4096_traffic.md",
               ["paper_2601_06849_gb300/csrc/gemm_tc.cu", "paper_2601_06849_gb300/csrc/tc_ptx.cuh",
                "paper_2601_06849_gb300/csrc/etd_internal.cuh"]),
    "fp64split": ("profiles/ozaki_pass_fp64split_fhn4096_traffic.md",
                  ["paper_2601_06849_gb300/csrc/ozaki.cu", "paper_2601_06849_gb300/csrc/tc_ptx.cuh",
                   "paper_2601_06849_gb300/csrc/etd_internal.cuh"]),
}
L2_BYTES = 129e6


def run_adjoint(args, world, rank, local):
    """Gradient workload: one timed iteration = forward solve over the window
    (checkpoints every 20 steps) + loss + backward through the library's adjoint
    steps (each segment recomputes its forward states on the device)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2601_06849_gb300 import autograd as AG
    from paper_2601_06849_gb300 import etd, inputs

    __graft_entry__.build()
    torch.cuda.set_device(local)
    d, n, ku, kv, q, tau, rx, desc = WORKLOADS[args.workload]
    window, every = 400, 20
    fdt = torch.float64 if args.precision in F64_PRECISIONS else torch.float32  # the plan's field type
    u0 = torch.tensor(inputs.fhn_uniform(n, d, workload=4), dtype=fdt, device="cuda")
    target = u0.clone()
    tplan = etd.Plan(d, n, ku * (1 + 1e-2), q, tau, precision=args.precision, reaction="fhn", rx_params=FHN, n_comp=2,
                     kappa_comp=(ku * (1 + 1e-2), kv))
    tplan.step(target, window)
    tplan.sync()
    tplan.close()

    u0_host = u0.cpu().pin_memory()

    def iteration(src=None):
        # src: pinned host copy of the initial field (the end-to-end leg copies it in)
        u0_ = (u0.clone() if src is None else src.to("cuda", non_blocking=True)).requires_grad_(True)
        kap = torch.tensor([ku, kv], dtype=torch.float64, requires_grad=True)
        rp = torch.tensor(FHN, dtype=torch.float64, requires_grad=True)
        u = AG.solve(u0_, kap, rp, d=d, n=n, q=q, dt=tau, n_steps=window, precision=args.precision, reaction="fhn",
                     checkpoint_every=every)
        loss = ((u - target) ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        return float(loss), kap.grad.clone(), rp.grad.clone()

    iters = max(1, min(args.steps, 3))
    for _ in range(args.warmup):
        iteration()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for _ in range(iters):
            loss, gk, gr = iteration()
        el = time.perf_counter() - t0
    el_max = barrier_max(el, world)
    # end to end: the initial field copied in from pinned host memory, loss and
    # gradients read back, every iteration
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        iteration(u0_host)
    el_e2e = barrier_max(time.perf_counter() - t0, world)
    unknowns = 2 * n ** d
    value = world * unknowns * window * iters / el_max
    # transform flops of an iteration: forward (4d passes per step), the recomputed
    # forward and the adjoint's 9 transforms (d passes each) per step, 2 n^(d+1) per
    # pass and component, times the split products
    products = {"fp64": 1, "fp32": 1, "tf32": 1, "tf32x3": 3, "bf16x3": 3, "bf16x6": 6, "tf32x6": 6,
                "fp64split": 21, "fp64split40": 15, "fp64split32": 10}.get(
        args.precision, 1)
    passes = window * (4 * d + 4 * d + 9 * d)
    flops = passes * 2.0 * n ** (d + 1) * 2 * products * iters
    peaks, src = measured_peaks()
    tpeak, tsrc = tensor_peak(peaks, src, args.precision, el_max)
    achieved = flops / el_max / 1e12
    line = {
        "metric": "unknown-updates/s per ETD2RK-DS step (forward + adjoint)", "value": value,
        "unit": "unknown-updates/s", "n_gpus": world, "steps": iters, "warmup": args.warmup,
        "ms_per_step": el_max / iters / window * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE.get(args.precision, args.precision),
        "data": "synthetic",
        "config": {"workload": desc, "d": d, "n": n, "window": window, "checkpoint_every": every,
                   "precision": args.precision, "step": "one forward + backward solve over the window",
                   "l2": "working set > 129 MB L2 (fields, checkpoints, adjoint workspace): no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": tpeak, "unit": "TFLOP/s",
                     "frac": achieved / tpeak, "traffic": None,
                     "kernel": "all transform passes of forward, recomputed forward and adjoint (whole-iteration rate)",
                     "peak_source": tsrc},
        # per time step: forward (2 reactions + 4d passes), the segment's recomputed
        # forward (the same), the adjoint step (9 transforms of 1 + d launches, 4
        # spectral combinations, 2 Jacobian products, 2 gradient reductions)
        "gpu_launches": iters * window * (2 * (2 + 4 * d) + 9 * (1 + d) + 8),
        "e2e": {"value": world * unknowns * window * iters / el_e2e, "unit": "unknown-updates/s",
                "h2d_bytes_per_step": 4 * unknowns, "d2h_bytes_per_step": 4 + 8 * 6,
                "per": "iteration (one forward + backward over the window)",
                "api": "torch.autograd through autograd.solve, initial field from pinned host memory, "
                       "loss and gradients read back"},
        "loss": loss, "grad_kappa": [float(x) for x in gk], "grad_rx": [float(x) for x in gr],
    }
    cs = clocks.summary()
    if cs:
        line["clocks"] = cs
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import adjoint as OA
        from oracle import oracle as O

        steps = 3
        P = O.Problem(d=d, n=n, kappa=(ku, kv), q=q, tau=tau, reaction="fhn", rp=FHN)
        x0 = u0.double().cpu().numpy()
        t0 = time.perf_counter()
        OA.adjoint_run(P, x0, steps, np.ones_like(x0))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": unknowns * steps / dt, "unit": "unknown-updates/s", "cores": O.max_threads(),
                                "kind": "oracle", "sample": f"FP64 NumPy adjoint oracle, {steps} forward + {steps} "
                                                            f"adjoint steps of the same 3D problem", "seconds": dt}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ensemble(args, world, rank, local):
    """Batched workload: one etd_batch_step per timed step over all instances."""
    import torch

    import __graft_entry__
    from paper_2601_06849_gb300 import etd, inputs

    __graft_entry__.build()
    torch.cuda.set_device(local)
    d, _, _, kv, q, _, rx, desc = WORKLOADS[args.workload]
    members = inputs.fhn_ensemble(512, workload=3)
    stream = torch.cuda.Stream()
    batch = etd.Batch(2, [m.n for m in members], [m.kappa_u for m in members], [q] * len(members),
                      [m.tau for m in members], precision=args.precision, reaction="fhn", rx_params=FHN, n_comp=2,
                      kappa_v=kv, stream=stream, autotune=args.autotune)
    info = batch.info()
    with torch.cuda.stream(stream):
        fields = [torch.tensor(m.u0, dtype=batch.dtype, device="cuda") for m in members]
        batch.step(fields, args.warmup)
        batch.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clocks:
            ev0.record(stream)
            batch.step(fields, args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        barrier(world)
        el_ms = ev0.elapsed_time(ev1)
        batch.sync()
    el_max = barrier_max(el_ms, world)
    value = world * info.unknowns * args.steps / (el_max / 1e3)
    # end to end: pinned host fields copied in, stepped, copied out, every step
    hosts = [torch.tensor(m.u0, dtype=batch.dtype).pin_memory() for m in members]
    e2e_steps = args.e2e_steps or 3
    with torch.cuda.stream(stream):
        dev = [h.to("cuda", non_blocking=True) for h in hosts]
        batch.step(dev, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for h, dv in zip(hosts, dev):
                dv.copy_(h, non_blocking=True)
            batch.step(dev, 1)
            for h, dv in zip(hosts, dev):
                h.copy_(dv, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = barrier_max(time.perf_counter() - t0, world)
    peaks, src = measured_peaks()
    flops = info.step_flops * max(info.products, 1) * args.steps
    sec = el_max / 1e3
    tpeak, tsrc = tensor_peak(peaks, src, args.precision, sec)
    tens = {"achieved": flops / sec / 1e12, "peak": tpeak, "unit": "TFLOP/s", "frac": flops / sec / 1e12 / tpeak,
            "peak_source": tsrc}
    sbytes = info.step_bytes * args.steps
    hbm = {"achieved": sbytes / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": sbytes / sec / 1e9 / peaks["hbm_gbs"], "peak_source": f"{src}: hbm_gbs"}
    bound = "hbm" if sbytes / (peaks["hbm_gbs"] * 1e9) > flops / (tpeak * 1e12) else "tensor"
    top = hbm if bound == "hbm" else tens
    nbytes = sum(h.numel() * h.element_size() for h in hosts)
    line = {
        "metric": "unknown-updates/s per ETD2RK-DS step", "value": value, "unit": "unknown-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.precision} (f32 fields, double-float spectral state)", "data": "synthetic",
        "config": {"workload": desc, "instances": len(members), "unknowns": info.unknowns,
                   "autotuned": bool(args.autotune),
                   "precision": args.precision, "pade": "P02",
                   "l2": f"working set {info.workspace_bytes / 1e9:.2f} GB > 129 MB L2: no flush",
                   "parallelism": f"replicas x{world}; groups by grid on concurrent streams, one CUDA graph per step"},
        "roofline": {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                     "frac": top["frac"], "traffic": None,
                     "kernel": "all transform passes of the ensemble over the timed region (whole-GPU rate)",
                     "peak_source": top["peak_source"], "tensor": tens, "hbm": hbm},
        "gpu_launches": args.steps * sum(10 for _ in range(15)),
        "e2e": {"value": world * info.unknowns * e2e_steps / e2e_s, "unit": "unknown-updates/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                "api": "etd.Batch.step on device copies of pinned host fields, 1 step per call"},
    }
    cs = clocks.summary()
    if cs:
        line["clocks"] = cs
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the timed fields went through warmup + steps steps: the FP64 oracle on
        # the first member of each grid size, from the same FP32-held input
        import numpy as np

        from oracle import oracle as O

        steps = args.warmup + args.steps
        errs, t0 = [], time.perf_counter()
        for i in ensemble_sample(members):
            m = members[i]
            P = O.Problem(d=2, n=m.n, kappa=(m.kappa_u, kv), q=q, tau=m.tau, reaction="fhn", rp=FHN)
            u0f = m.u0.astype(np.float32).astype(np.float64) if batch.dtype == torch.float32 else m.u0
            errs.append(max(rel_errs(fields[i].double().cpu().numpy(), O.run(P, u0f, steps))))
        dt = time.perf_counter() - t0
        line["rel_err_vs_fp64_oracle"] = max(errs)
        line["cpu_baseline"] = {"value": sum(2 * members[i].n ** 2 for i in ensemble_sample(members)) * steps / dt,
                                "unit": "unknown-updates/s", "cores": O.max_threads(), "kind": "oracle",
                                "sample": f"{steps} FP64 oracle steps of the first member of each of the "
                                          f"{len(errs)} grid sizes", "seconds": dt}
    batch.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def rel_errs(got, ref):
    """max |got - ref| / max |ref| per component over the whole field (the error metric)."""
    import numpy as np

    return [float(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max()) for c in range(ref.shape[0])]


def ensemble_sample(members):
    """Indices of the ensemble members whose error is checked: the first member
    of each grid size (all 15 sizes of the workload, 64 .. 512)."""
    seen, idx = set(), []
    for i, m in enumerate(members):
        if m.n not in seen:
            seen.add(m.n)
            idx.append(i)
    return idx


def run_accuracy(args, world, rank, local):
    """--accuracy: the error of each precision against the FP64 oracle over the
    configuration's whole run length (checked at every tenth of the run, the
    largest of those errors reported), beside two floors that no FP32-field path
    can beat: the FP64 oracle run from the unrounded FP64 draw of u0 against the
    one from its FP32 rounding (one FP32 rounding of the input, amplified by the
    dynamics), and the oracle's FP32 shadow (the same LU scheme in FP32
    arithmetic). FP32 paths are compared with the oracle run from the same
    FP32-held input; the FP64 path with the one from the FP64 draw."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import __graft_entry__
    from oracle import oracle as O
    from paper_2601_06849_gb300 import etd, inputs

    __graft_entry__.build()
    torch.cuda.set_device(local)
    name = args.workload
    total = args.accuracy_steps or RUN_STEPS[name]
    marks = sorted(set(max(1, total * (i + 1) // 10) for i in range(10)))
    precisions = [x for x in args.precisions.split(",") if x]
    O.lib()
    if name == "ensemble512":
        members = inputs.fhn_ensemble(512, workload=3)
        sample = ensemble_sample(members)
        d, _, _, kv, q, _, rx, desc = WORKLOADS[name]

        def oracle_runs(src):  # checkpoints of every sampled member
            out = []
            for i in sample:
                m = members[i]
                P = O.Problem(d=2, n=m.n, kappa=(m.kappa_u, kv), q=q, tau=m.tau, reaction="fhn", rp=FHN)
                u, prev, cps = src(m), 0, []
                for k in marks:
                    u = O.run(P, u, k - prev)
                    cps.append(u)
                    prev = k
                out.append(cps)
            return out
        t0 = time.perf_counter()
        ref32 = oracle_runs(lambda m: m.u0.astype(np.float32).astype(np.float64))
        ref64 = oracle_runs(lambda m: m.u0)
        oracle_s = time.perf_counter() - t0
        floor_in = [max(max(rel_errs(a[j], b[j])) for a, b in zip(ref64, ref32)) for j in range(len(marks))]
        floor_sh = [0.0] * len(marks)
        for si, i in enumerate(sample):
            m = members[i]
            P = O.Problem(d=2, n=m.n, kappa=(m.kappa_u, kv), q=q, tau=m.tau, reaction="fhn", rp=FHN)
            u, prev = m.u0.astype(np.float32).astype(np.float64), 0
            for j, k in enumerate(marks):
                u = O.run(P, u, k - prev, precision="f32").astype(np.float64)
                floor_sh[j] = max(floor_sh[j], max(rel_errs(u, ref32[si][j])))
                prev = k
        errors = {}
        for prec in precisions:
            batch = etd.Batch(2, [m.n for m in members], [m.kappa_u for m in members], [q] * len(members),
                              [m.tau for m in members], precision=prec, reaction="fhn", rx_params=FHN, n_comp=2,
                              kappa_v=kv)
            ref = ref64 if prec in F64_PRECISIONS else ref32
            fields = [torch.tensor(m.u0, dtype=batch.dtype, device="cuda") for m in members]
            prev, per = 0, []
            for j, k in enumerate(marks):
                batch.step(fields, k - prev)
                batch.sync()
                prev = k
                per.append(max(max(rel_errs(fields[i].double().cpu().numpy(), ref[si][j]))
                               for si, i in enumerate(sample)))
            errors[prec] = {"max": max(per), "final": per[-1], "per_checkpoint": per}
            batch.close()
        line = {"metric": "max rel err vs FP64 oracle over the run", "workload": desc, "steps": total,
                "checkpoints": marks, "sampled_instances": [{"index": i, "n": members[i].n} for i in sample],
                "errors": errors,
                "floors": {"fp32_input_rounding": {"max": max(floor_in), "per_checkpoint": floor_in},
                           "fp32_shadow": {"max": max(floor_sh), "per_checkpoint": floor_sh}},
                "oracle": {"seconds": oracle_s, "cores": O.max_threads()},
                "error_metric": "max over checkpoints, components and sampled instances of "
                                "max|U - U_ref| / max|U_ref|"}
        print(json.dumps(line), flush=True)
        return
    d, n, ku, kv, q, tau, rx, desc = WORKLOADS[name]
    kap = (ku, kv) if rx == "fhn" else (ku,)
    P = O.Problem(d=d, n=n, kappa=kap, q=q, tau=tau, pade=2, reaction=rx, rp=FHN if rx == "fhn" else ())
    u0 = initial_field(name)
    u0f = u0.astype(np.float32).astype(np.float64)  # the values an FP32 field holds

    def oracle_checkpoints(u, precision="f64"):
        out, prev = [], 0
        for k in marks:
            u = O.run(P, u, k - prev, t0=prev * tau, precision=precision)
            out.append(np.asarray(u, dtype=np.float64))
            prev = k
        return out
    need32 = args.floors or any(pr not in F64_PRECISIONS for pr in precisions)
    need64 = args.floors or any(pr in F64_PRECISIONS for pr in precisions)
    t0 = time.perf_counter()
    ref32 = oracle_checkpoints(u0f) if need32 else None
    ref64 = oracle_checkpoints(u0) if need64 else None
    oracle_s = (time.perf_counter() - t0) / (int(need32) + int(need64))
    floor_in = [max(rel_errs(a, b)) for a, b in zip(ref64, ref32)] if args.floors else None
    floor_sh = ([max(rel_errs(a, b)) for a, b in zip(oracle_checkpoints(u0f, "f32"), ref32)]
                if args.floors else None)
    errors = {}
    for prec in precisions:
        plan = make_plan(name, prec)
        ref = ref64 if prec in F64_PRECISIONS else ref32
        x = torch.tensor(u0, dtype=plan.dtype, device="cuda")
        prev, per = 0, []
        t0 = time.perf_counter()
        for j, k in enumerate(marks):
            plan.step(x, k - prev)
            plan.sync()
            prev = k
            per.append(max(rel_errs(x.double().cpu().numpy(), ref[j])))
        errors[prec] = {"max": max(per), "final": per[-1], "per_checkpoint": per,
                        "seconds": time.perf_counter() - t0}
        plan.close()
    line = {"metric": "max rel err vs FP64 oracle over the run", "workload": desc, "steps": total,
            "checkpoints": marks, "errors": errors,
            "floors": ({"fp32_input_rounding": {"max": max(floor_in), "per_checkpoint": floor_in},
                        "fp32_shadow": {"max": max(floor_sh), "per_checkpoint": floor_sh}} if args.floors else None),
            "oracle": {"seconds_per_run": oracle_s, "cores": O.max_threads()},
            "error_metric": "max over checkpoints and components of max|U - U_ref| / max|U_ref|"}
    print(json.dumps(line), flush=True)


def initial_field(name):
    from paper_2601_06849_gb300 import inputs

    d, n, ku, kv, q, tau, rx, _ = WORKLOADS[name]
    if rx == "fhn":
        return inputs.fhn_uniform(n, d, workload=1)
    if d == 3:
        return inputs.gaussian_bump(n, 3)
    return inputs.allen_cahn_2d(n, workload=0)


def make_plan(name, precision, stream=None, autotune=False):
    from paper_2601_06849_gb300 import etd

    d, n, ku, kv, q, tau, rx, _ = WORKLOADS[name]
    if rx == "fhn":
        return etd.Plan(d, n, ku, q, tau, pade=2, precision=precision, reaction="fhn", rx_params=FHN, n_comp=2,
                        kappa_comp=(ku, kv), stream=stream, autotune=autotune)
    return etd.Plan(d, n, ku, q, tau, pade=2, precision=precision, reaction=rx, n_comp=1, stream=stream,
                    autotune=autotune)


def tensor_peak(peaks, src, precision, timed_s):
    """Tensor peak for the precision's product kind: the measured BF16 burst rate
    for a timed region shorter than 2 s (the kernels run near the burst clocks),
    the sustained rate for longer ones; TF32 products at the nominal TF32/BF16
    ratio of it."""
    key = "bf16_tflops" if timed_s < 2.0 else "bf16_tflops_sustained"
    bf16_mode = precision.startswith("bf16") or precision.startswith("fp64split")  # the slices are BF16
    peak = peaks[key] * (1.0 if bf16_mode else TF32_OVER_BF16)
    return peak, f"{src}: {key}" + ("" if bf16_mode else " x 1.1/2.25 (TF32/BF16 nominal)")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier_max(value, world):
    """Barrier, then the max of `value` over ranks."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def cpu_baseline(name, gpu_field=None, gpu_steps=0, max_steps=200, fp32_input=True, min_seconds=12.0):
    """The FP64 CPU oracle as it stands, all host cores, on the same workload.

    It runs min(gpu_steps, max_steps) time steps (at least 5) from the same
    initial field (as the GPU received it: rounded to FP32 for the FP32-field
    precisions); when that covers every step the GPU took, the GPU's field is
    compared with the oracle's (max |U_gpu - U_oracle| / max |U_oracle| per
    component, the error the metric is quoted at). Then it continues, timed
    only, until about min_seconds of CPU work (or max_steps) make the sample."""
    import numpy as np

    from oracle import oracle as O

    d, n, ku, kv, q, tau, rx, _ = WORKLOADS[name]
    kap = (ku, kv) if rx == "fhn" else (ku,)
    P = O.Problem(d=d, n=n, kappa=kap, q=q, tau=tau, pade=2, reaction=rx, rp=FHN if rx == "fhn" else ())
    u0 = initial_field(name)
    if fp32_input:
        u0 = u0.astype(np.float32).astype(np.float64)
    O.lib()  # build and load before timing
    steps = max(5, min(gpu_steps, max_steps))
    t0 = time.perf_counter()
    ref = O.run(P, u0, steps)
    dt = time.perf_counter() - t0
    # a sample of about min_seconds of CPU work: further steps from the compared
    # field (timed only; the workloads' reactions do not depend on t)
    total = steps
    more = ref
    while dt < min_seconds and total < max_steps:
        chunk = min(max(1, steps // 3), max_steps - total)
        t1 = time.perf_counter()
        more = O.run(P, more, chunk)
        dt += time.perf_counter() - t1
        total += chunk
    out = {"value": u0.size * total / dt, "unit": "unknown-updates/s", "cores": O.max_threads(), "kind": "oracle",
           "sample": f"{total} FP64 time steps of the full {name} workload ({u0.size} unknowns), the first {steps} "
                     f"compared with the GPU's field; Thomas/LU oracle, OpenMP over 1D lines", "seconds": dt}
    if gpu_field is not None and steps == gpu_steps:
        err = [float(np.abs(gpu_field[c] - ref[c]).max() / np.abs(ref[c]).max()) for c in range(ref.shape[0])]
        out["rel_err_vs_gpu"] = max(err)
        out["rel_err_per_component"] = err
    return out


def recorded_traffic(kernel_files, record):
    """Bytes per launch from a committed ncu record, if the kernel sources still
    hash to what was profiled; else None."""
    import hashlib

    h = hashlib.sha256()
    for f in kernel_files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    try:
        with open(os.path.join(ROOT, record)) as fh:
            rec = dict(line.strip().split(": ", 1) for line in fh if ": " in line and not line.startswith("#"))
    except OSError:
        return None, h.hexdigest()
    if rec.get("kernel_source_sha256") != h.hexdigest():
        return None, h.hexdigest()
    return float(rec["dram_bytes_per_launch"]), h.hexdigest()


def run_reference(args, world, rank):
    """--impl reference: the FP64 CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from oracle import oracle as O

    name = args.workload
    d, n, ku, kv, q, tau, rx, desc = WORKLOADS[name]
    kap = (ku, kv) if rx == "fhn" else (ku,)
    u0 = initial_field(name)
    # per-step sample: one full time step of the workload, unless the whole run
    # would exceed ~150 s; then the same workload on a coarser grid.
    P = O.Problem(d=d, n=n, kappa=kap, q=q, tau=tau, pade=2, reaction=rx, rp=FHN if rx == "fhn" else ())
    t0 = time.perf_counter()
    O.run(P, u0, 1)
    one = time.perf_counter() - t0
    sample_n = n
    budget = 150.0
    while (args.steps + args.warmup) * one > budget and sample_n > 256:
        sample_n //= 2
        one /= (2 ** (d + 1))
    if sample_n != n:
        P = O.Problem(d=d, n=sample_n, kappa=kap, q=q, tau=tau, pade=2, reaction=rx, rp=P.rp)
        from paper_2601_06849_gb300 import inputs

        u0 = inputs.fhn_uniform(sample_n, d, workload=1) if rx == "fhn" else (
            inputs.gaussian_bump(sample_n, 3) if d == 3 else inputs.allen_cahn_2d(sample_n, workload=0))
    u = O.run(P, u0, args.warmup)
    t0 = time.perf_counter()
    u = O.run(P, u, args.steps)
    el = time.perf_counter() - t0
    value = u.size * args.steps / el
    sample = (f"each step: one FP64 oracle time step of {name}" +
              (f" on the coarser n={sample_n} grid" if sample_n != n else " (full grid)"))
    line = {"impl": "reference", "metric": "unknown-updates/s per ETD2RK-DS step", "value": value,
            "unit": "unknown-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": sample_n, "d": d, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "unknown-updates/s", "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "unknown-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="fhn2d_4096", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64split")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="time the pass kernel candidates at plan creation")
    ap.add_argument("--accuracy", action="store_true",
                    help="error vs the FP64 oracle over the workload's whole run length, with floors")
    ap.add_argument("--precisions", default="bf16x6,tf32x3", help="--accuracy: comma-separated precisions")
    ap.add_argument("--accuracy-steps", type=int, default=None, help="--accuracy: override the run length")
    ap.add_argument("--no-floors", dest="floors", action="store_false",
                    help="--accuracy: skip the FP32-shadow and input-rounding floors (two oracle runs fewer)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.accuracy:
        run_accuracy(args, world, rank, local)
        return

    if args.workload == "ensemble512":
        run_ensemble(args, world, rank, local)
        return
    if args.workload == "adjoint3d_128":
        run_adjoint(args, world, rank, local)
        return

    import torch

    import __graft_entry__
    from paper_2601_06849_gb300 import etd

    __graft_entry__.build()
    torch.cuda.set_device(local)
    name = args.workload
    d, n, ku, kv, q, tau, rx, desc = WORKLOADS[name]
    stream = torch.cuda.Stream()
    plan = make_plan(name, args.precision, stream=stream, autotune=args.autotune)
    info = plan.info()
    u0 = initial_field(name)
    u = torch.tensor(u0, dtype=plan.dtype, device="cuda")
    with torch.cuda.stream(stream):
        plan.step(u, args.warmup)
        plan.sync()
        plan.set_timing(True)
        for kind in (0, 1, 2):
            plan.kernel_times(kind)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clocks:
            ev0.record(stream)
            plan.step(u, args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        barrier(world)
        el_ms = ev0.elapsed_time(ev1)
        plan.sync()
        gemm_ms, gemm_n = plan.kernel_times(0)
        rx_ms, rx_n = plan.kernel_times(1)
        acc_ms, acc_n = plan.kernel_times(2)
        plan.set_timing(False)
    el_max = barrier_max(el_ms, world)
    m, bad = plan.stats(u)
    unknowns = info.unknowns
    value = world * unknowns * args.steps / (el_max / 1e3)

    # end to end through the public host entry point: H2D + step + D2H each step
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 10))
    host = torch.tensor(u0, dtype=plan.dtype).pin_memory()
    plan.step_host(host, 1)  # warm the host path
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.step_host(host, 1)
    e2e_s = barrier_max(time.perf_counter() - t0, world)
    bytes_field = unknowns * (8 if plan.dtype == torch.float64 else 4)

    gpu_field = u.double().cpu().numpy()
    peaks, src = measured_peaks()
    avg_gemm_ms = gemm_ms / max(gemm_n, 1)
    if info.products > 0:
        # one per-step transform pass: its algorithmic flops and DRAM bytes, and
        # the bound whose time is larger (2D m=4096: tensor; 3D m=256: HBM)
        flops = info.gemm_flops * info.products
        bytes_pass = info.step_bytes / info.gemms_per_step
        tpeak, tsrc = tensor_peak(peaks, src, args.precision, el_max / 1e3)
        hpeak = peaks["hbm_gbs"]
        sec = avg_gemm_ms * 1e-3
        tens = {"achieved": flops / sec / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                "frac": flops / sec / 1e12 / tpeak, "per_launch": flops, "peak_source": tsrc}
        hbm = {"achieved": bytes_pass / sec / 1e9, "peak": hpeak, "unit": "GB/s",
               "frac": bytes_pass / sec / 1e9 / hpeak, "per_launch": bytes_pass, "peak_source": f"{src}: hbm_gbs"}
        bound = "hbm" if bytes_pass / (hpeak * 1e9) > flops / (tpeak * 1e12) else "tensor"
        top = hbm if bound == "hbm" else tens
        traffic, src_hash = (None, None)
        if name == "fhn2d_4096" and args.precision in TRAFFIC_RECORDS:
            record, files = TRAFFIC_RECORDS[args.precision]
            traffic, src_hash = recorded_traffic(files, record)
        roof = {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                "frac": top["frac"], "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "kernel": ("FP64-split transform pass (oz_slice_kernel + ozaki_pass_kernel, tcgen05 BF16 slice "
                           "products), per-step passes, mean over the step" if args.precision.startswith("fp64split") else
                           "tcgen05 transform pass (per-step passes, mean over the step)"),
                "peak_source": top["peak_source"], "avg_launch_ms": avg_gemm_ms,
                "tensor": tens, "hbm": hbm}
    elif args.precision == "dst32":
        # fast sine transform passes (row FFTs in shared memory + a transposing
        # epilogue): HBM against the pass's algorithmic bytes (operand in, result
        # and carried state out; the row kernel's scratch round trip is not counted)
        bytes_pass = info.step_bytes / info.gemms_per_step
        hpeak = peaks["hbm_gbs"]
        achieved = bytes_pass / (avg_gemm_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hpeak, "unit": "GB/s", "frac": achieved / hpeak,
                "traffic": None, "kernel": "fast sine transform pass (dst_rows_kernel + dst_transpose_epi_kernel)",
                "peak_source": f"{src}: hbm_gbs", "avg_launch_ms": avg_gemm_ms, "bytes_per_launch": bytes_pass}
    else:
        flops = info.gemm_flops
        lanes = 128 if plan.dtype == torch.float32 else 2  # FP32 lanes / FP64 units per SM
        clk = 2.07e9
        peak = 152 * lanes * 2 * clk / 1e12
        achieved = flops / (avg_gemm_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "gemm_simt_kernel (transform pass)",
                "peak_source": "152 SMs x FMA lanes x 2 x 2.07 GHz", "flops_per_launch": flops,
                "avg_launch_ms": avg_gemm_ms}

    line = {
        "metric": "unknown-updates/s per ETD2RK-DS step",
        "value": value,
        "unit": "unknown-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": el_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE.get(args.precision, args.precision),
        "data": "synthetic",
        "config": {"workload": desc, "d": d, "n": n, "n_comp": info.n_comp, "precision": args.precision,
                   "pass_kernel": {"persistent": list(info.pass_persistent), "tile_n": list(info.pass_tile_n),
                                   "autotuned": bool(args.autotune)},
                   "pade": "P02", "unknowns": unknowns,
                   "l2": f"working set {info.workspace_bytes / 1e9:.2f} GB > 129 MB L2: inputs larger than L2, no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        # every kernel launch of the timed steps: the passes and reaction kernels the
        # plan's per-launch timing events counted (reactions fused into the pass
        # epilogues add none), times the kernels one pass launches
        "gpu_launches": (gemm_n + acc_n) * info.kernels_per_pass + rx_n,
        "kernel_ms": {"transform_passes": gemm_ms, "transform_launches": gemm_n, "reaction_ms": rx_ms,
                      "reaction_launches": rx_n, "accurate_transform_ms": acc_ms, "accurate_transform_launches": acc_n},
        "e2e": {"value": world * unknowns * e2e_steps / e2e_s, "unit": "unknown-updates/s",
                "h2d_bytes_per_step": bytes_field, "d2h_bytes_per_step": bytes_field,
                "steps": e2e_steps, "api": "etd_step_host (pinned host field, 1 step per call)"},
        "field_max_abs": m,
        "nonfinite": bad,
    }
    cs = clocks.summary()
    if cs:
        line["clocks"] = cs
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, gpu_field, args.warmup + args.steps,
                                            fp32_input=plan.dtype == torch.float32)
        if "rel_err_vs_gpu" in line["cpu_baseline"]:
            line["rel_err_vs_fp64_oracle"] = line["cpu_baseline"]["rel_err_vs_gpu"]
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
