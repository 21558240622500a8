#!/usr/bin/env python
"""Exact lnL evaluations per second at N_model = 11,424 on one GB300.

Workload: three sub-band instruments on one uv grid (n_f = 24, 32, 48
channels; N_model = 6048, 7840, 11424; 331 baselines x 16 times), B = 16
prior points each, all 48 factorised in one batched evaluation (one graph
launch).  A step is one such evaluation.  The headline counts only the 16
evaluations at N_model = 11,424 per step (the smaller sub-bands ride along
and are reported separately: the whole mix, and each sub-band timed alone).
The mixed-precision path is timed; the float64 GPU path is timed on one
point per sub-band for the comparison, and the CPU oracle on one
N_model = 11,424 evaluation for the host baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own replica of the workload
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SUBBANDS = ("C3_24", "C3_32", "C3_48")
WORKLOADS = {"c3": SUBBANDS, "c1": ("C1",)}
METRIC = ("exact lnL evals/s at N_model=11424 (C3 sub-band mix, mixed precision; only the 11424-mode "
          "evaluations of each batched step are counted)")
HEADLINE = "C3_48"
UNIT = "evals/s"
# bf16 tensor operations of one trailing-update output tile (128 x 64 complex,
# K = 128 complex): per K-chunk and A part (Im, Re) the products' N sum to
# 1920 columns for the full slice-pair set (diagonal tiles; 15 pairs) and to
# 1408 for the reduced one (off-diagonal tiles; 11 pairs), each column
# 2 * 128 * 16 flops: 2 parts x 8 K-chunks x N x 4096
TILE_TENSOR_FLOP_FULL = 2 * 8 * 1920 * 2 * 128 * 16
TILE_TENSOR_FLOP_REDUCED = 2 * 8 * 1408 * 2 * 128 * 16
TILE_USEFUL_FLOP = 8 * 128 * 64 * 128      # the complex GEMM it computes


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def build_workload(B: int, names=SUBBANDS):
    from synth import build_instrument, draw_phi
    insts = {}
    if "C3_48" in names:
        insts["C3_48"] = build_instrument("C3_48")
        for name in ("C3_24", "C3_32"):
            insts[name] = build_instrument(name, A_from=insts["C3_48"])
    for name in names:
        if name not in insts:
            insts[name] = build_instrument(name)
    phis = {n: draw_phi(insts[n].spec, B) for n in names}
    return insts, phis


def make_likes(P, insts, precision, names=SUBBANDS):
    likes = []
    for n in names:
        inst = insts[n]
        lk = P.Likelihood(precision)
        lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
        lk.set_data(inst.d, inst.noise_var)
        lk.precompute()
        likes.append(lk)
    return likes


def trail_tiles_per_step(n_models, B):
    """Trailing-update tiles of one batched evaluation (all problems, all
    steps): (all tiles, tiles on the diagonal of their block step's update)."""
    tot, diag = 0, 0
    for n in n_models:
        nt = (n + 127) // 128
        for k in range(nt - 1):
            T = nt - k - 1
            tot += B * T * (T + 1)   # T(T+1)/2 block pairs x 2 column halves
            diag += B * T * 2
    return tot, diag


def cpu_baseline(insts):
    """The oracle, as it stands, on the host cores: one evaluation of the
    N_model = 11,424 sub-band (its precompute of M is not timed)."""
    import oracle as O
    from synth import draw_phi
    inst = insts[HEADLINE]
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    phi = draw_phi(inst.spec, 1, stream=9)[0]
    t0 = time.perf_counter()
    O.evaluate(M, db, inst.kbin, phi, inst.spec.lssm_prior_var)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one oracle evaluation at N_model={inst.spec.n_model} ({dt:.1f} s; numpy/BLAS threads "
                      "use the host cores), precompute of M not timed"}


def workload_config(workload, B, n_models):
    """The `config` object of the bench line, the same for both arms."""
    if workload == "c3":
        name = ("C3: 3 sub-band instruments (n_f 24/32/48, N_model 6048/7840/11424, "
                "331 baselines x 16 times), B=%d each, one batched evaluation per step" % B)
    else:
        name = "C1: one instrument (N_model 3280, 126 baselines x 19 times x 38 channels), B=%d" % B
    # double-float working matrices: lower-triangle 128-tiles, 16 bytes per complex element
    ws_bytes = sum(B * (nt * (nt + 1) // 2) * 128 * 128 * 16 for nt in ((n + 127) // 128 for n in n_models))
    return {"workload": name, "B_per_subband": B, "n_model": list(n_models),
            "l2": "inputs larger than L2 (working matrices %.1f GB)" % (ws_bytes / 1e9), "parallelism": "replicas"}


def run_reference(args):
    """The oracle on the host cores, on this arm's metric: each step is one
    oracle evaluation at N_model = 6048 (about 3 s), converted to
    evaluations per second at N_model = 11,424 by the cubic cost of the
    Cholesky, (11424/6048)^3 = 6.74, so that the whole run stays within a
    few minutes (one evaluation at 11,424 takes about 20 s)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    insts, _ = build_workload(1)
    n_models = [insts[n].spec.n_model for n in SUBBANDS]
    import oracle as O
    inst = insts["C3_24"]
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    from synth import draw_phi
    phis = draw_phi(inst.spec, args.warmup + args.steps, stream=9)
    for p in phis[: args.warmup]:
        O.evaluate(M, db, inst.kbin, p, inst.spec.lssm_prior_var)
    t0 = time.perf_counter()
    for p in phis[args.warmup:]:
        O.evaluate(M, db, inst.kbin, p, inst.spec.lssm_prior_var)
    dt = (time.perf_counter() - t0) / args.steps
    scale = (insts[HEADLINE].spec.n_model / inst.spec.n_model) ** 3
    value = 1.0 / (dt * scale)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config("c3", args.B, n_models),
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": value,
                             "sample": f"one oracle evaluation at N_model={inst.spec.n_model} per step "
                                       f"({dt:.2f} s), scaled to N_model=11424 by the cubic cost (x{scale:.2f})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--B", type=int, default=16)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true", help="skip the two-batches-in-flight measurement")
    ap.add_argument("--no-tune", action="store_true", help="default schedule instead of the autotuner's")
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS),
                    help="c3: the sub-band mix (default); c1: the 3280-mode instrument (small profiling case)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_2501_12928_gb300 as P

    names = WORKLOADS[args.workload]
    insts, phis = build_workload(args.B, names)
    n_models = [insts[n].spec.n_model for n in names]
    t0 = time.perf_counter()
    likes = make_likes(P, insts, "mixed", names)
    torch.cuda.synchronize()
    t_pre = time.perf_counter() - t0
    # schedule of this batch shape: the autotuner's choice (cached per box in the build folder)
    tune = None
    if not args.no_tune:
        t0 = time.perf_counter()
        tune = P.autotune(likes, [phis[n] for n in names], reps=2,
                          cache_path=os.path.join(ROOT, "paper_2501_12928_gb300", "_build", "schedule_cache.jsonl"))
        tune["seconds"] = round(time.perf_counter() - t0, 1)
    stream = torch.cuda.current_stream()
    dev_phi = [torch.tensor(phis[n], dtype=torch.float64, device="cuda") for n in names]
    out = [torch.empty(args.B, dtype=torch.float64, device="cuda") for _ in names]
    sts = [torch.empty(args.B, dtype=torch.int32, device="cuda") for _ in names]
    P.set_profiling(True)

    def step():
        _lnl_multi_dev(P, likes, dev_phi, out, sts)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    trail_ms, trail_n, cls_ms = 0.0, 0, {}
    gap_any, gap_main, ms_eval = 0.0, 0.0, 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
            st = likes[0].stats()
            trail_ms += st["ms_class"]["trail"]
            trail_n += st["n_class"]["trail"]
            for k, v in st["ms_class"].items():
                cls_ms[k] = cls_ms.get(k, 0.0) + v
            if st["ms_busy_any"] >= 0:
                ms_eval += st["ms_last"]
                gap_any += st["ms_last"] - st["ms_busy_any"]
                gap_main += st["ms_last"] - st["ms_busy_main"]
        e1.record(stream)
        torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1) / 1e3
    if dist:
        from paper_2501_12928_gb300.replicas import max_over_ranks
        elapsed = max_over_ranks(elapsed)
    evals_step = args.B * len(names)
    # headline: the evaluations at the largest model dimension of each step
    head_step = args.B if HEADLINE in names else evals_step
    value = head_step * args.steps * ws / elapsed
    mix_value = evals_step * args.steps * ws / elapsed
    launches = likes[0].stats()["kernel_launches"]
    status_ok = all(int((s != 0).sum().item()) == 0 for s in sts)

    # end to end through the public API with host buffers (copies inside the timed region)
    P.set_profiling(False)
    host_phi = [np.ascontiguousarray(phis[n]) for n in names]
    for _ in range(2):
        P.lnl_multi(likes, host_phi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        outs, _ = P.lnl_multi(likes, host_phi)
    t_e2e = time.perf_counter() - t0
    e2e_value = head_step * args.steps * ws / t_e2e

    # each sub-band alone (B points, one batched evaluation per step), for the per-size rates
    per_subband = None
    if len(names) > 1:
        per_subband = {}
        for n, lk, dp, o, sst in zip(names, likes, dev_phi, out, sts):
            one = lambda: _lnl_multi_dev(P, [lk], [dp], [o], [sst])   # noqa: E731
            for _ in range(2):
                one()
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            k_one = max(2, min(args.steps, 5))
            a0.record(stream)
            for _ in range(k_one):
                one()
            a1.record(stream)
            torch.cuda.synchronize()
            t1 = a0.elapsed_time(a1) / 1e3 / k_one
            per_subband[str(insts[n].spec.n_model)] = {"value": args.B / t1, "unit": UNIT,
                                                      "ms_per_step": t1 * 1e3, "B": args.B}

    # two batches in flight: asynchronous calls on slots 0 and 1 and two
    # streams, so that one batch's latency-bound last block steps overlap the
    # next batch's heavy steps (an extra field; `value` above is one batch at a time)
    two = None
    if not args.no_pipeline:
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        o2 = [[torch.empty(args.B, dtype=torch.float64, device="cuda") for _ in names] for _ in range(2)]
        s2 = [[torch.empty(args.B, dtype=torch.int32, device="cuda") for _ in names] for _ in range(2)]
        Bs = [args.B] * len(names)
        for _ in range(2):
            for slot in (0, 1):
                P.lnl_multi_async(likes, dev_phi, o2[slot], s2[slot], slot, streams[slot])
                P.lnl_multi_wait(likes, Bs, slot, streams[slot])
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event()
        a0.record(streams[0])
        streams[1].wait_event(a0)
        for i in range(args.steps):
            slot = i % 2
            P.lnl_multi_async(likes, dev_phi, o2[slot], s2[slot], slot, streams[slot])
        b1.record(streams[1])
        streams[0].wait_event(b1)
        a1.record(streams[0])
        for slot in (0, 1):
            P.lnl_multi_wait(likes, Bs, slot, streams[slot])
        t2 = a0.elapsed_time(a1) / 1e3
        if dist:
            t2 = max_over_ranks(t2)
        ok2 = all(int((x != 0).sum().item()) == 0 for q in s2 for x in q)
        two = {"value": evals_step * args.steps * ws / t2, "unit": UNIT, "ms_per_step": t2 / args.steps * 1e3,
               "slots": 2, "status_all_ok": ok2, "counts": "every evaluation of the mix (%d per batch)" % evals_step,
               "how": "beor_lnl_multi_async on two slots and two streams, device buffers, CUDA events"}

    # roofline of the dominant kernel (trailing slice GEMM), timed inside the steps above
    peaks, peak_src = _peaks()
    tiles, diag_tiles = trail_tiles_per_step(n_models, args.B)
    tensor_flop = diag_tiles * TILE_TENSOR_FLOP_FULL + (tiles - diag_tiles) * TILE_TENSOR_FLOP_REDUCED
    trail_s = trail_ms / 1e3 / args.steps
    # achieved: the method's own work (the complex GEMM of every trailing tile,
    # 8 real flops per complex multiply-add) per second of trailing-kernel time;
    # tc_achieved: the bf16 tensor operations the slice products perform
    useful = tiles * TILE_USEFUL_FLOP / trail_s / 1e12 if trail_s > 0 else None
    performed = tensor_flop / trail_s / 1e12 if trail_s > 0 else None
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    burst = peaks.get("bf16_tflops", 1900.0)
    traffic = _traffic_per_launch(tiles / max(1, trail_n / args.steps))
    roof = {"bound": "tensor", "achieved": useful, "peak": peak, "unit": "TFLOP/s",
            "frac": useful / peak if useful else None, "traffic": traffic,
            "kernel": "slice_gemm_kernel<TRAIL>: trailing update of the blocked complex Cholesky",
            "achieved_is": "complex GEMM flops of the trailing update (8 per complex multiply-add) / kernel time",
            "peak_source": f"bf16 dense sustained, {peak_src}",
            "frac_burst": useful / burst if useful else None,
            "tc_achieved": performed, "tc_frac": performed / peak if performed else None,
            "tc_is": "bf16 tensor operations of the exact slice products (%d per diagonal tile, %d per other "
                     "tile)" % (TILE_TENSOR_FLOP_FULL, TILE_TENSOR_FLOP_REDUCED),
            "avg_launch_ms": trail_ms / max(1, trail_n)}

    # float64 GPU comparator: one point per sub-band in one batched evaluation
    fp64 = None
    if not args.no_fp64:
        P.set_profiling(False)
        lf = make_likes(P, insts, "fp64", names)
        ph1 = [phis[n][:1] for n in names]
        P.lnl_multi(lf, ph1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.fp64_steps):
            P.lnl_multi(lf, ph1)
        dt = (time.perf_counter() - t0) / args.fp64_steps
        fp64 = {"value": len(names) / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
                "workload": "one point per sub-band (N 6048/7840/11424) per batched evaluation"}
        for lk in lf:
            lk.close()

    cpu = None
    if rank == 0 and not args.no_cpu and args.workload == "c3":
        cpu = cpu_baseline(insts)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 slice products (exact, fp32 accumulate) + double-float / f64",
            "data": "synthetic",
            "config": dict(workload_config(args.workload, args.B, n_models), precompute_s=round(t_pre, 2)),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * sum(p.size for p in host_phi),
                    "d2h_bytes_per_step": 12 * evals_step},
            "gpu_launches": int(launches) * args.steps,
            "roofline": roof,
            "cpu_baseline": cpu,
            "mix": {"value": mix_value, "unit": UNIT, "evals_per_step": evals_step,
                    "flop_weighted_11424_equiv": (mix_value / evals_step) * sum(
                        args.B * (n / 11424.0) ** 3 for n in n_models)},
            "per_subband": per_subband,
            "fp64_gpu": fp64,
            "two_in_flight": two,
            "speedup_vs_fp64_gpu": mix_value / fp64["value"] if fp64 else None,
            "schedule": tune,
            "kernel_ms_per_step": {k: v / args.steps for k, v in cls_ms.items()},
            "graph_gaps": {"ms_per_step": ms_eval / args.steps,
                           "ms_no_kernel_in_flight": gap_any / args.steps,
                           "ms_main_stream_idle": gap_main / args.steps,
                           "how": "union of every launch's interval between the CUDA events that bracket it "
                                  "inside the graph; the rest of the evaluation has no kernel launched and "
                                  "unfinished on any stream (main stream alone: second figure)"},
            "status_all_ok": status_ok,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _lnl_multi_dev(P, likes, dev_phi, out, sts):
    """One batched evaluation with device-resident inputs and outputs."""
    import ctypes
    from paper_2501_12928_gb300 import beor as Bm
    n = len(likes)
    ctxs = (ctypes.c_void_p * n)(*[lk._h.value for lk in likes])
    pp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in dev_phi])
    Bs = (ctypes.c_int * n)(*[t.shape[0] for t in dev_phi])
    op = (ctypes.c_void_p * n)(*[t.data_ptr() for t in out])
    sp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in sts])
    import torch
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Bm._check(Bm._lib().beor_lnl_multi(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(pp, ctypes.c_void_p),
                                       ctypes.cast(Bs, ctypes.c_void_p), ctypes.cast(op, ctypes.c_void_p),
                                       ctypes.cast(sp, ctypes.c_void_p), s), "beor_lnl_multi")


def _traffic_per_launch(tiles_per_launch):
    """DRAM bytes per trailing launch from the committed ncu summary, if any:
    the per-tile DRAM bytes measured on the 3280-mode case (traffic per tile
    is the working-matrix read-modify-write, the same at every size) times
    the tiles of an average launch."""
    path = os.path.join(ROOT, "profiles", "slice_gemm_trail_C1_B8.md")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("dram_bytes_per_tile:"):
                    return float(line.split(":")[1]) * tiles_per_launch
    except OSError:
        pass
    return None


if __name__ == "__main__":
    main()
