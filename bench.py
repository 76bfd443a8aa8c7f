#!/usr/bin/env python
"""Benchmark of the MPS-LCC hot path on GB300.

One step = one two-site LCC sweep (left -> right -> left over all positions)
of the first-order wavefunction: at every position the transition right-hand
side (P1^T H Phi0), the overlap projection, the local linear solve built on
the sigma vector (H0_eff - E0) x, the FP64 Hylleraas value, the truncation and
the three environment renormalisations.  The DMRG reference (Davidson
sweeps) and the MPO build are set-up work and run before the timed region.

Default workload: 3-band Hubbard model, 2x4 cells (24 orbitals, 9 up + 9 down
holes), reference M0 = 500, first-order M1 = 2000, tensor-core sigma products
(BF16 operands, FP32 accumulation) with FP64 residuals.

Printed metric: sigma-vector TFLOP/s over the timed sweeps (algorithmic flops
of every sigma product divided by the device time of the whole sweeps), plus
the sweep seconds and the energies.  ``--impl reference`` times the CPU oracle
instead (see ``cpu_sample``).
"""
from __future__ import annotations

import argparse
import json
import pickle
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "bf16x3": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--M0", type=int, default=None)
    ap.add_argument("--M1", type=int, default=None)
    ap.add_argument("--dmrg-sweeps", type=int, default=8)
    ap.add_argument("--dmrg-init", choices=["product", "random"], default="product",
                    help="reference start: lowest-h_pp determinant or random MPS")
    ap.add_argument("--prec", default="bf16x3", choices=list(PREC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--save-state", default=None,
                    help="after the timed steps, write the reference and first-order MPS to this file")
    ap.add_argument("--load-state", default=None,
                    help="start from states written by --save-state instead of the reference sweeps "
                         "(used to profile the timed sweep without the set-up)")
    ap.add_argument("--fp64-sweep", action="store_true",
                    help="also time one sweep on the plain FP64 path from the same states (about 8 minutes "
                         "at M1 = 2000)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile-sigma", type=int, default=0,
                    help="profiling mode: N sigma products at the middle position inside NVTX range 'sigma'")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d.get("hbm_gbs", 6800.0), bf16=d.get("bf16_tflops", 1900.0),
                    bf16_sust=d.get("bf16_tflops_sustained", 1700.0), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sust=1700.0, src="fallback")


# FP64 pipe of GB300 (nominal, no FP64 tensor path): 1.25 TFLOP/s
FP64_PEAK_TFLOPS = 1.25


class Clocks:
    """nvidia-smi sampler over the timed region."""

    def __init__(self, device):
        self.device = device
        self.proc = None
        # samples go to $MPSLCC_CLOCKS_DIR (default: the system temp directory)
        self.out = os.path.join(os.environ.get("MPSLCC_CLOCKS_DIR", tempfile.gettempdir()),
                                f"mpslcc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.out), exist_ok=True)
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.out).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].strip().lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows)}


def cpu_sample(budget_s):
    """Time the CPU oracle's local problem: sigma = P^T H0 P psi built densely
    in the determinant space (Implementation section, Fig. 3).  The oracle
    holds at most ~10^4 determinants, so the sample is the L=8 chain
    workload (4900 determinants, a random M=64 first-order MPS) rather than
    the 24-orbital workload; flops are counted with the library's sigma
    accounting for the same local problem."""
    import numpy as np

    import synth
    from oracle import fci, mps as omps
    c = synth.config(0)
    dets = fci.determinants(8, 4, 4)
    H = fci.build_hamiltonian(c["h"], c["V"], dets)
    H0 = fci.fink_h0(H, dets, 8, c["n_core"], c["n_active"])
    m = synth.random_mps(8, 8, 0, M=64, seed=5)
    l = 3
    n = len(omps.local_layout(m, l)[0])
    psi = synth.random_vector(n, 1)
    t0 = time.perf_counter()
    steps = 0
    while True:
        Heff = omps.effective_hamiltonian(m, l, H0, dets)
        _ = Heff @ psi
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / steps
    return dict(seconds_per_sigma=dt, steps=steps, n_local=n, mps=m, l=l)


def sigma_flops_host(mps, l, mpo_class_sizes):
    """Library's algorithmic flop count of one sigma (two phases) for bra =
    ket = mps at position l; mpo_class_sizes maps the class quantum-number
    change (dN, d2Sz) to the number of channels on the middle MPO bond."""
    LQ = [(0, 0), (1, 1), (1, -1), (2, 0)]

    def fl(bond, mask):
        d = {}
        for s in mask:
            for (n, sz, dim) in bond:
                q = (n + LQ[s][0], sz + LQ[s][1])
                d[q] = d.get(q, 0) + dim
        return d

    def fr(mask, bond):
        d = {}
        for s in mask:
            for (n, sz, dim) in bond:
                q = (n - LQ[s][0], sz - LQ[s][1])
                d[q] = d.get(q, 0) + dim
        return d

    FL = fl(mps["bonds"][l], mps["masks"][l])
    FR = fr(mps["masks"][l + 1], mps["bonds"][l + 2])
    mid = [q for q in FL if q in FR]
    f = 0.0
    for qb in mid:
        K = 0
        for dq, nw in mpo_class_sizes.items():
            qk = (qb[0] - dq[0], qb[1] - dq[1])
            if qk in FL and qk in FR:
                K += nw * FL[qk]
                f += 2.0 * nw * FR[qb] * FL[qk] * FR[qk]
        f += 2.0 * FL[qb] * FR[qb] * K
    return f


def workload_config(c, M0, M1, world):
    return {"workload": c["name"], "n_orb": c["n_orb"], "n_elec": c["n_alpha"] + c["n_beta"],
            "n_core": c["n_core"], "n_active": c["n_active"], "M0": M0, "M1": M1,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "working set (environments, fused operators) far above L2"}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    import paper_1509_00216_gb300 as mp  # host-only context: MPO class sizes for the flop count
    import synth
    wc = synth.config(args.config)
    c = synth.config(0)
    ctx = mp.Context(device=-1)
    ctx.build_mpo(c["h"], c["V"], 8, 0)
    ctx.set_spaces(c["n_core"], c["n_active"])
    idx, _ = None, None
    s = None
    times = []
    for i in range(args.warmup + args.steps):
        s = cpu_sample(max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup)))
        if i >= args.warmup:
            times.append(s["seconds_per_sigma"])
    # class sizes of the H0 MPO on the middle bond of position l
    classes = _mpo_classes(ctx, mp.MPO_H0, s["l"] + 1)
    ctx.close()
    f = sigma_flops_host(s["mps"], s["l"], classes)
    dt = sum(times) / len(times)
    v = f / dt / 1e12
    cores = os.cpu_count()
    line = dict(metric=METRIC, value=v, unit="TFLOP/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=dt * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=workload_config(wc, args.M0 or wc["M0"], args.M1 or wc["M1"], world),
                cpu_baseline={"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                              "sample": "dense determinant-space P^T H0 P psi at position 3 of a random "
                                        "M=64 MPS of the L=8 chain (4900 determinants): the oracle cannot "
                                        "hold the 24-orbital workload, so this local sigma stands in for it; "
                                        "flops = library sigma accounting"},
                e2e={"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    print(json.dumps(line), flush=True)


def _mpo_classes(ctx, which, bond):
    """Channel counts per quantum-number class of one MPO bond (from the
    exported site tensor's right channels)."""
    import numpy as np
    idx, val = ctx.export_mpo_site(which, bond - 1)
    LQ = [(0, 0), (1, 1), (1, -1), (2, 0)]
    # propagate channel QN changes from the left boundary
    k = ctx.n_orb
    dq = {0: (0, 0)}
    for p in range(bond):
        ii, _ = ctx.export_mpo_site(which, p)
        nd = {}
        for (w0, w1, so, si) in ii:
            if w0 in dq and w1 not in nd:
                a = dq[w0]
                nd[w1] = (a[0] + LQ[so][0] - LQ[si][0], a[1] + LQ[so][1] - LQ[si][1])
        dq = nd
    out = {}
    for w, q in dq.items():
        out[q] = out.get(q, 0) + 1
    return out


SIGMA_TRAFFIC_RATIO = (3.270 + 3.547) / (2.512 + 2.690)
METRIC = "sigma-vector TFLOP/s and LCC sweep s at M=2000, mixed vs FP64; |dE| vs oracle"


def gpu_arm(args, rank, world, local_rank):
    import torch

    import paper_1509_00216_gb300 as mp
    import synth

    dist = world > 1
    if dist:
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    c = synth.config(args.config)
    M0 = args.M0 or c["M0"]
    M1 = args.M1 or c["M1"]
    prec = PREC[args.prec]
    ctx = mp.Context(device=local_rank, prec=prec, tol=1e-8, max_iter=60, torch_memory=True,
                     init_guess=1 if args.dmrg_init == "product" else 0)
    ctx.build_mpo(c["h"], c["V"], c["n_alpha"] + c["n_beta"], 0)
    ctx.set_spaces(c["n_core"], c["n_active"])
    if args.load_state:
        with open(args.load_state, "rb") as f:
            saved = pickle.load(f)
        ctx.load_mps(0, saved["phi0"])
        E0 = ctx.dmrg_reference(M0, 0)
        ctx.load_mps(1, saved["phi1"])
    else:
        E0 = ctx.dmrg_reference(M0, args.dmrg_sweeps)
    for _ in range(args.warmup):
        ctx.lcc_sweep(M1, 1)
    stream = torch.cuda.current_stream()
    if args.profile_sigma:
        # profiling mode: repeated sigma products at the middle position of
        # the converged state, inside the NVTX range "sigma" (for ncu filters)
        l = c["n_orb"] // 2 - 1
        n_out, n_in = ctx.local_dim(l, mp.OP_H0_11)
        x = torch.randn(n_in, dtype=torch.float64, device="cuda")
        y = torch.empty(n_out, dtype=torch.float64, device="cuda")
        ctx.apply_heff_device(l, mp.OP_H0_11, x.data_ptr(), y.data_ptr(), n_in, n_out, prec)
        ctx.reset_stats()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("sigma")
        for _ in range(args.profile_sigma):
            ctx.apply_heff_device(l, mp.OP_H0_11, x.data_ptr(), y.data_ptr(), n_in, n_out, prec)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        st = ctx.stats()
        print(json.dumps({"profile_sigma": args.profile_sigma, "site": l, "n_local": n_in,
                          "tc_phase1_s": st["tc_phase1_seconds"], "tc_phase2_s": st["tc_phase2_seconds"],
                          "tc_phase1_bytes": st["tc_phase1_bytes"], "tc_phase2_bytes": st["tc_phase2_bytes"],
                          "sigma_flops": st["sigma_flops"], "calls": st["sigma_calls"]}), flush=True)
        ctx.close()
        return
    ctx.reset_stats()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        torch.cuda.nvtx.range_push("timed")
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.lcc_sweep(M1, 1)      # E2 (8 bytes) is read back to the host by every call
        ev1.record(stream)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
    if dist:
        td.barrier()
    dev_s = ev0.elapsed_time(ev1) * 1e-3
    st = ctx.stats()
    flops = st["sigma_flops"]
    flops2 = flops
    e = ctx.energy()
    if dist:
        t = torch.tensor([dev_s, e2e_s], device="cuda")
        td.all_reduce(t, op=td.ReduceOp.MAX)
        dev_s, e2e_s = t.tolist()
    pk = peaks()
    kern = st["sigma_seconds"]
    if prec == 0:
        # FP64 DFMA path: ALU-bound against the FP64 pipe
        roof = {"bound": "alu", "achieved": flops / kern / 1e12 if kern else None, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "kernel": "gemm_f64_kernel (sigma phases)"}
    else:
        # tensor-core sigma GEMMs run at ~55 flop/byte, far below the BF16
        # ridge (~250): they are bounded by HBM bandwidth.  Algorithmic bytes
        # = operands read once + results written (hi + lo pieces in split mode)
        tcs = st["tc_phase1_seconds"] + st["tc_phase2_seconds"]
        tcb = st["tc_phase1_bytes"] + st["tc_phase2_bytes"]
        launches = max(1, st["tc_launches"])
        roof = {"bound": "hbm", "achieved": tcb / tcs / 1e9 if tcs else None, "peak": pk["hbm"], "unit": "GB/s",
                "kernel": "tc_gemm_kernel (both sigma phases)", "launches": st["tc_launches"],
                "bytes_per_launch": tcb / launches, "us_per_launch": tcs / launches * 1e6,
                "phase1_gbs": st["tc_phase1_bytes"] / st["tc_phase1_seconds"] / 1e9 if st["tc_phase1_seconds"] else None,
                "phase2_gbs": st["tc_phase2_bytes"] / st["tc_phase2_seconds"] / 1e9 if st["tc_phase2_seconds"] else None,
                "tensor_tflops": flops / tcs / 1e12 if tcs else None,
                "tensor_frac_of_bf16_sustained": flops / tcs / 1e12 / pk["bf16_sust"] if tcs else None}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] else None
    if prec != 0:
        # DRAM bytes per algorithmic byte of the sigma launches, from one ncu
        # capture of both phases at the middle position of the 3-band workload
        # at M1 = 1000 (3.270 + 3.547 GB against 2.512 + 2.690 GB); the traffic
        # of a launch scales with the bytes it moves, so the full-size figure
        # is this ratio times the algorithmic bytes per launch
        roof["traffic"] = SIGMA_TRAFFIC_RATIO * roof["bytes_per_launch"]
        roof["traffic_source"] = "ncu dram bytes ratio 1.31 at M1=1000, scaled to the launch's algorithmic bytes"
    else:
        roof["traffic"] = None
    roof["peak_source"] = pk["src"]
    value = world * flops / dev_s / 1e12
    line = dict(metric=METRIC, value=value, unit="TFLOP/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=dev_s / args.steps * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={0: "f64", 1: "tf32", 2: "bf16", 3: "bf16x3"}[prec], data="synthetic",
                config=workload_config(c, M0, M1, world),
                sweep_s=dev_s / args.steps, sigma_calls=st["sigma_calls"], sigma_kernel_s=kern,
                stage_s={k: st[k] for k in ("t_plan", "t_rhs", "t_solve", "t_trunc", "t_env", "t_fuse_left", "t_fuse_right", "t_tc_prepare")},
                fused_ahead={"used": st["ahead_used"], "missed": st["ahead_missed"]},
                energies={k: e[k] for k in ("E0", "E2", "E3", "E_lcc2", "E_lcc3", "max_discarded_weight")},
                roofline=roof, gpu_launches=st["kernel_launches"],
                e2e={"value": world * flops2 / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                     "d2h_bytes_per_step": 8})
    clk_s = clk.summary()
    if clk_s:
        line["clocks"] = clk_s
    if args.save_state:
        with open(args.save_state, "wb") as f:
            pickle.dump({"phi0": ctx.export_mps(0), "phi1": ctx.export_mps(1)}, f, protocol=4)
    if args.fp64_sweep and prec != 0:
        # the same sweep on the plain FP64 path (DFMA GEMMs), from the same
        # reference and first-order states, outside the timed region
        p0, p1 = ctx.export_mps(0), ctx.export_mps(1)
        ctx.close()
        c64 = mp.Context(device=local_rank, prec=mp.FP64, tol=1e-8, max_iter=60, torch_memory=True)
        c64.build_mpo(c["h"], c["V"], c["n_alpha"] + c["n_beta"], 0)
        c64.set_spaces(c["n_core"], c["n_active"])
        c64.load_mps(0, p0)
        c64.dmrg_reference(M0, 0)
        c64.load_mps(1, p1)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        c64.lcc_sweep(M1, 1)
        f1.record(stream)
        torch.cuda.synchronize()
        f64_s = f0.elapsed_time(f1) * 1e-3
        c64.close()
        line["fp64_sweep_s"] = f64_s
        line["sweep_speedup_vs_fp64"] = f64_s / (dev_s / args.steps)
    ctx.close()
    if rank == 0:
        if not args.no_cpu_baseline:
            s = cpu_sample(args.cpu_seconds)
            hc = mp.Context(device=-1)
            c0 = synth.config(0)
            hc.build_mpo(c0["h"], c0["V"], 8, 0)
            hc.set_spaces(c0["n_core"], c0["n_active"])
            cls = _mpo_classes(hc, mp.MPO_H0, s["l"] + 1)
            hc.close()
            f = sigma_flops_host(s["mps"], s["l"], cls)
            line["cpu_baseline"] = {"value": f / s["seconds_per_sigma"] / 1e12, "unit": "TFLOP/s",
                                    "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"{s['steps']} dense P^T H0 P psi on the L=8 chain local problem "
                                              f"(n_local={s['n_local']}); the oracle cannot hold 24 orbitals"}
        print(json.dumps(line), flush=True)
    if dist:
        td.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        reference_arm(args, rank, world)
    else:
        gpu_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
