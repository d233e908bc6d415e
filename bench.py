#!/usr/bin/env python
"""Throughput benchmark of the FE-P3M library: particles/s for Phi_i + forces.

Workload: the jittered rock-salt lattice, 32^3 = 32,768 ions (+/-1 on a simple
cubic grid of spacing L/32, each coordinate jittered by U[-1e-3, 1e-3] L,
seed 2), on a periodic 32^3-element mesh (q = 1, p = 3, 7^3 short-range block).
One step = set_particles (binning) + compute(Phi, U, forces) through the C ABI:
assembly, forward multigrid solve, pair kernel, energy, adjoint solve and
reverse sweeps.  The headline is the mixed-precision path; the FP64 path is
timed beside it.  Inputs are far smaller than L2, so a 256 MB buffer is written
between timed steps (L2 flush, untimed).

--impl reference times the CPU oracle (the plain FP64 implementation) on the
same workload.  With torchrun (N > 1) every rank runs an independent replica
(the method is not sharded across GPUs in this build); rank 0 prints.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/sec for Phi_i+forces at stated RMS error vs Ewald; mixed vs FP64; % roofline"
WORKLOAD = "nacl32"
GOLDEN = os.path.join(ROOT, "tests", "golden", "nacl32_sample.txt")
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one k_pair_screen launch and of one transform pass of the
# mesh solve (k_tc_rows, both right-hand sides) on this workload, from the ncu captures summarised in
# profiles/ (None until one is taken of the current kernel)
PAIR_DRAM_BYTES = 2264320 + 1536
PASS_DRAM_BYTES = 7187200 + 0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--large", type=int, default=1,
                   help="1: also time the water (999 999 atoms, 128^3) and clustered (4e6, 256^3) workloads")
    p.add_argument("--legs", default="all", choices=["all", "main"],
                   help="main: only the timed loop of --precision (no FP64 leg, end-to-end leg or accuracy); "
                        "for profiling")
    p.add_argument("--workload", default=WORKLOAD,
                   help="with --legs main: the workload of the timed loop (nacl32, uniform262k, water1m, ...)")
    p.add_argument("--profile-step", action="store_true",
                   help="bracket the last timed step with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    return p.parse_args()


def replica_throughput(total_ms, units, steps, ws, device):
    """Whole-job throughput of ws independent replicas that each processed `units` per step for `steps`
    steps: the job's time is the slowest rank's (MAX over ranks).  Returns (job ms, units per second)."""
    if ws > 1:
        import torch
        import torch.distributed as tdist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, ws * units * steps / (total_ms / 1e3)


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_golden():
    U = None
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("# U_fep3m_oracle"):
                U = float(line.split()[-1])
    a = np.loadtxt(GOLDEN)
    return dict(idx=a[:, 0].astype(int), phi_e=a[:, 1], F_e=a[:, 2:5], phi_o=a[:, 5], F_o=a[:, 6:9], U_o=U)


def rel_rms(x, ref, shift=False):
    d = x - ref
    if shift:
        d = d - d.mean()       # potentials are compared up to a constant (Sec. 4)
    return float(np.linalg.norm(d) / np.linalg.norm(ref))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def fp32_peak_tflops(n_sm, mhz):
    # FP32 FMA: 128 lanes per SM, 2 flops per FMA
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


def time_engine(eng, pos, Q, out, steps, warmup, flush, torch, host=False, profile_last=False):
    """Run warmup + timed steps; returns (ms per step, (screen-kernel ms, inner-solve ms) per step, launches per
    step, the last result).  With timing enabled on eng, the stage times of each step are kept in eng.step_stats.
    profile_last: the last step between cudaProfilerStart and cudaProfilerStop."""
    stream = eng.stream
    for _ in range(warmup):
        eng.set_particles(pos, Q)
        eng.compute(phi=True, energy=True, forces=True, out=out)
    torch.cuda.synchronize()
    l0 = eng.stats()["kernel_launches"]
    ms, pair = [], []
    for k in range(steps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        if profile_last and k == steps - 1:
            torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        eng.set_particles(pos, Q)
        r = eng.compute(phi=True, energy=True, forces=True, out=out)
        e1.record(stream)
        e1.synchronize()
        if profile_last and k == steps - 1:
            torch.cuda.profiler.stop()
        ms.append(e0.elapsed_time(e1))
        st = eng.stats()
        pair.append((st["ms_pair_screen"], st["ms_inner_solve"]))
        eng.step_stats.append(st)
    launches = (eng.stats()["kernel_launches"] - l0) / steps
    return ms, pair, launches, r


STAGES = ("ms_bin", "ms_assemble", "ms_solve", "ms_inner_solve", "ms_pair_screen", "ms_pair_eval", "ms_adjoint")


def large_workload(name, steps, warmup, flush, dev, torch, peaks):
    """One of the full-size workloads (mixed, forces), timed like the headline: particles/s, per-step
    stage times (CUDA events on their streams; the stages overlap across the four streams) and the
    roofline of the two largest kernels: the transform pass of the mesh solve (tensor pipe: 2 N flops per
    node and mode column and right-hand side, six split-bf16 products) and the short-range screen kernel
    (FP32: 1024 flops per non-empty target element and non-empty element of its block, 20 per singular
    pair)."""
    from paper_1503_08509_gb300 import api, workloads
    d = workloads.workload(name)
    N = len(d["Q"])
    pos = torch.tensor(d["pos"], device=dev)
    Q = torch.tensor(d["Q"], device=dev)
    eng = api.FEP3M(d["L"], d["n_el"], precision="mixed", device=dev.index)
    eng.set_timing(True)
    eng.step_stats = []
    out = dict(phi=torch.empty(N, dtype=torch.float64, device=dev),
               forces=torch.empty((N, 3), dtype=torch.float64, device=dev))
    ms, pair, launches, r = time_engine(eng, pos, Q, out, steps, warmup, flush, torch)
    st = eng.stats()
    stages = {k: round(statistics.mean(x[k] for x in eng.step_stats), 3) for k in STAGES}
    Nn = 3 * d["n_el"]
    pass_ms = stages["ms_inner_solve"] / 6
    nrhs = st["solve_rhs"]                  # the step pairs the forward and adjoint right-hand sides
    pass_flops = 2.0 * Nn ** 4 * 6          # six split products per pass and right-hand side
    # the same inner solve alone on the GPU (fep3m_solve_mesh of a random neutral load): in the step it
    # shares the GPU with the concurrent adjoint solve and the short-range kernels
    rhs = torch.randn(Nn ** 3, dtype=torch.float64, device=dev)
    rhs -= rhs.mean()
    alone = []
    for _ in range(3):
        eng.solve_mesh(rhs)
        alone.append(eng.stats()["ms_inner_solve"])
    del rhs
    alone_ms = statistics.median(alone[1:]) / 6
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    props = torch.cuda.get_device_properties(dev)
    fp32 = fp32_peak_tflops(props.multi_processor_count, peaks.get("sm_max_mhz", 2070.0))
    flops_elem = st["screen_element_pairs"] * 1024 + st["singular_pairs"] * 20
    pair_ms = stages["ms_pair_screen"]
    res = {"workload": name, "n": N, "n_el": d["n_el"], "steps": steps, "warmup": warmup,
           "value": round(N * steps / (sum(ms) / 1e3), 1), "unit": "particles/s",
           "ms_per_step": round(sum(ms) / steps, 3), "stages_ms": stages,
           "gpu_launches": int(round(launches)),
           "mg": {"refine_steps": st["refine_steps"], "rel_residual": st["mg_rel_residual"],
                  "adj_rel_residual": st["adj_rel_residual"]},
           "pairs": {"singular": st["singular_pairs"], "screen_element_pairs": st["screen_element_pairs"],
                     "nonempty_elements": st["nonempty_elements"], "max_per_element": st["max_per_element"]},
           "roofline_transform": {"kernel": "k_tc_rows (transform pass of the mesh solve)", "bound": "tensor",
                                  "achieved": round(nrhs * pass_flops / (pass_ms * 1e-3) / 1e12, 1),
                                  "peak": bf16, "unit": "TFLOP/s",
                                  "frac": round(nrhs * pass_flops / (pass_ms * 1e-3) / 1e12 / bf16, 4),
                                  "count": "2 N^4 x 6 split-bf16 products per pass and right-hand side, N = %d, "
                                           "%d right-hand sides per pass in the step (1 alone)" % (Nn, nrhs),
                                  "ms_per_launch": round(pass_ms, 4),
                                  "peak_note": "measured sustained bf16 (MEASURED_PEAKS.json)",
                                  "alone": {"ms_per_launch": round(alone_ms, 4),
                                            "achieved": round(pass_flops / (alone_ms * 1e-3) / 1e12, 1),
                                            "frac": round(pass_flops / (alone_ms * 1e-3) / 1e12 / bf16, 4),
                                            "note": "the forward solve's first inner solve by fep3m_solve_mesh, "
                                                    "no concurrent streams; frac of the sustained peak"}},
           "roofline_pair": {"kernel": "k_pair_screen", "bound": "alu",
                             "achieved": round(flops_elem / (pair_ms * 1e-3) / 1e12, 2), "peak": round(fp32, 2),
                             "unit": "TFLOP/s", "frac": round(flops_elem / (pair_ms * 1e-3) / 1e12 / fp32, 4),
                             "ms_per_launch": pair_ms}}
    eng.close()
    del pos, Q, out
    torch.cuda.empty_cache()
    return res


def box_workload(kind, steps, warmup, flush, dev, torch):
    """The box with Dirichlet or Neumann data (Sec. "Alternate boundary conditions"), mixed, Phi and U:
    the rock-salt ions of the headline workload moved to the element centres (offset h/2, so that the
    jitter keeps every ion inside the box [0, L]^3), 32^3 box elements, grounded (g = 0) or zero-flux
    data.  particles/s of set_particles + compute(Phi, U)."""
    from paper_1503_08509_gb300 import api, workloads
    pos_np, Q_np = workloads.rock_salt(32, L=1.0, jitter=1e-3, seed=2, offset=0.5)
    N = len(Q_np)
    pos = torch.tensor(pos_np, device=dev)
    Q = torch.tensor(Q_np, device=dev)
    eng = api.FEP3M(1.0, 32, precision="mixed", device=dev.index, dirichlet=kind == "dirichlet",
                    neumann=kind == "neumann")
    out = dict(phi=torch.empty(N, dtype=torch.float64, device=dev))
    l0 = None
    ms = []
    for k in range(warmup + steps):
        if k == warmup:
            torch.cuda.synchronize()
            l0 = eng.stats()["kernel_launches"]
        flush.add_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(eng.stream)
        eng.set_particles(pos, Q)
        r = eng.compute(phi=True, energy=True, forces=False, out=out)
        e1.record(eng.stream)
        e1.synchronize()
        if k >= warmup:
            ms.append(e0.elapsed_time(e1))
    st = eng.stats()
    res = {"workload": "rock salt 32^3 ions at the element centres (jitter 1e-3 L) in a box of 32^3 elements, "
                       "%s data (%s)" % (kind, "g = 0" if kind == "dirichlet" else "zero flux"),
           "n": N, "steps": steps, "warmup": warmup, "value": round(N * steps / (sum(ms) / 1e3), 1),
           "unit": "particles/s", "ms_per_step": round(sum(ms) / steps, 3),
           "gpu_launches": int(round((st["kernel_launches"] - l0) / steps)),
           "mg": {"refine_steps": st["refine_steps"], "rel_residual": st["mg_rel_residual"]},
           "U": r["U"]}
    eng.close()
    return res


def run_ours(args):
    import torch
    ws, rank, local = dist()
    if ws > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1503_08509_gb300 import api, build, workloads
    build.build()
    d = workloads.workload(args.workload if args.legs == "main" else WORKLOAD)
    N = len(d["Q"])
    pos = torch.tensor(d["pos"], device=dev)
    Q = torch.tensor(d["Q"], device=dev)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    results = {}
    legs = [args.precision] + (["fp64"] if args.precision == "mixed" and args.legs == "all" else [])
    for prec in legs:
        eng = api.FEP3M(d["L"], d["n_el"], precision=prec, device=dev.index)
        eng.set_timing(True)
        eng.step_stats = []
        out = dict(phi=torch.empty(N, dtype=torch.float64, device=dev),
                   forces=torch.empty((N, 3), dtype=torch.float64, device=dev))
        main = prec == args.precision
        steps = args.steps if main else max(3, args.steps // 4)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else dev.index)
        if main:
            clocks.start()
        ms, pair, launches, r = time_engine(eng, pos, Q, out, steps, args.warmup, flush, torch,
                                            profile_last=main and args.profile_step)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ck = clocks.stop() if main else None
        total, _ = replica_throughput(sum(ms), N, steps, ws, dev)
        st = eng.stats()
        results[prec] = dict(ms=ms, total=total, steps=steps, pair=pair, launches=launches, stats=st, clocks=ck,
                             phi=out["phi"].cpu().numpy(), F=out["forces"].cpu().numpy(), U=r["U"], eng=eng)

    main = results[args.precision]
    value = ws * N * main["steps"] / (main["total"] / 1e3)   # total: already the slowest rank's
    if args.legs == "main":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 1), "unit": "particles/s", "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup, "legs": "main",
                              "workload": args.workload,
                              "ms_per_step": round(main["total"] / main["steps"], 4)}))
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # end to end through the public API with pinned host buffers (H2D inputs, D2H Phi/forces/U)
    eng = main["eng"]
    pos_h = torch.tensor(d["pos"]).pin_memory().numpy()
    Q_h = torch.tensor(d["Q"]).pin_memory().numpy()
    phi_h = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    F_h = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
    for _ in range(args.warmup):
        eng.set_particles(pos_h, Q_h)
        eng.compute(forces=True, out=dict(phi=phi_h, forces=F_h))
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eng.set_particles(pos_h, Q_h)
        eng.compute(forces=True, out=dict(phi=phi_h, forces=F_h))
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total, e2e_value = replica_throughput(sum(e2e_ms), N, args.steps, ws, dev)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # accuracy against the stored oracle / Ewald sample and between the two precisions
    g = load_golden()
    acc = {}
    for prec, rr in results.items():
        acc[prec] = dict(
            phi_rel_rms_vs_ewald=rel_rms(rr["phi"][g["idx"]], g["phi_e"], shift=True),
            force_rel_rms_vs_ewald=rel_rms(rr["F"][g["idx"]], g["F_e"]),
            phi_rel_rms_vs_oracle=rel_rms(rr["phi"][g["idx"]], g["phi_o"]),
            force_rel_rms_vs_oracle=rel_rms(rr["F"][g["idx"]], g["F_o"]),
            U_rel_vs_oracle=abs(rr["U"] - g["U_o"]) / abs(g["U_o"]))
    if "fp64" in results and args.precision == "mixed":
        acc["mixed_vs_fp64"] = dict(phi_rel_rms=rel_rms(results["mixed"]["phi"], results["fp64"]["phi"]),
                                    force_rel_rms=rel_rms(results["mixed"]["F"], results["fp64"]["F"]))

    st = main["stats"]
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)

    # roofline of the step's dominant kernel (the largest share of the step's launch time in the ncu launch
    # list): k_tc_rows, the tensor-core transform passes of the mesh solve.  Each pass reads and writes the
    # (3n)^3 FP32 vector once: 8 B per degree of freedom per fine-level sweep of the mesh solve.  Timed with
    # CUDA events recorded inside the replayed solve graph around the forward solve's first inner solve (six
    # passes), concurrent with the rest of the step.
    nodes = (3 * d["n_el"]) ** 3
    inner_ms = statistics.mean(p[1] for p in main["pair"])
    pass_ms = inner_ms / 6 if inner_ms > 0 else float("nan")
    hbm = peaks.get("hbm_gbs")
    hbm_note = "measured copy bandwidth (MEASURED_PEAKS.json)"
    if not hbm:
        hbm, hbm_note = 6800.0, "fallback 6.8 TB/s"
    rhs = st["solve_rhs"]   # right-hand sides per pass: the forward and adjoint solves go through together
    pass_bytes = 8 * nodes * rhs
    achieved_gbs = pass_bytes / (pass_ms * 1e-3) / 1e9
    roof = {"kernel": "k_tc_rows (fast-diagonalisation transform pass of the mesh solve, tensor cores)",
            "bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved_gbs / hbm, 4), "traffic": PASS_DRAM_BYTES, "peak_note": hbm_note,
            "count": "8 B per node and right-hand side per pass ((3n)^3 = %d nodes, FP32 read + write; %d "
                     "right-hand sides per pass)" % (nodes, rhs),
            "bytes_per_launch": pass_bytes, "ms_per_launch": round(pass_ms, 5),
            "note": "at 32^3 the vector (3.5 MB) stays in L2 and each pass is launch/latency bound"}

    # roofline of the short-range kernel the method is built around: k_pair_screen (FP32 issue bound),
    # timed with CUDA events on its own stream, where it runs concurrently with the forward and adjoint mesh
    # solves.  achieved = the algorithmic element-to-point count for a build that collapses the screen sums per
    # target element (1024 flops per non-empty target element and non-empty element of its block, 20 per
    # singular pair with gradients; the 128 per target of the 64-node evaluation belong to k_pair_eval);
    # the per-target-charge count and the flops the kernel executes (vertex-regrouped contraction: 512 x 64
    # x 2 per non-empty target element) are reported beside it.
    ne_nonempty = st["nonempty_elements"]
    pairs = st["singular_pairs"]
    flops_elem = st["screen_element_pairs"] * 1024 + pairs * 20
    flops_charge = st["screen_charge_pairs"] * 1024 + pairs * 20
    flops_exec = ne_nonempty * 512 * 64 * 2 + pairs * 20
    pair_ms = statistics.mean(p[0] for p in main["pair"])
    tf = lambda f: f / (pair_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    roof_pair = {"kernel": "k_pair_screen (screen-field contraction + singular pairs with gradients, concurrent "
                           "with the mesh solves)",
                 "bound": "alu", "achieved": round(tf(flops_elem), 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                 "frac": round(tf(flops_elem) / peak, 4), "traffic": PAIR_DRAM_BYTES,
                 "peak_note": "FP32 FMA peak derived: %d SMs x 128 lanes x 2 flops x %.0f MHz (max SM clock)"
                              % (props.multi_processor_count, sm_max),
                 "count": "per (non-empty target element, non-empty block element) pair x 1024 + singular pairs x 20",
                 "flops_per_launch": flops_elem, "ms_per_launch": round(pair_ms, 4),
                 "per_target_charge": {"flops": flops_charge, "frac": round(tf(flops_charge) / peak, 4)},
                 "executed": {"flops": flops_exec, "frac": round(tf(flops_exec) / peak, 4)}}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(main["total"] / main["steps"], 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": "jittered rock salt 32^3 = 32768 ions (+/-1, spacing L/32, jitter 1e-3 L), "
                               "periodic 32^3 hex mesh, q=1 (p=3), 7^3 short-range block",
                   "precision": args.precision, "step": "set_particles + compute(Phi, U, forces)",
                   "l2": "256 MB buffer written between timed steps (inputs < L2)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "accuracy": acc,
        "fp64": ({"value": round(ws * N * results["fp64"]["steps"] / (results["fp64"]["total"] / 1e3), 1),
                  "ms_per_step": round(results["fp64"]["total"] / results["fp64"]["steps"], 4)}
                 if "fp64" in results and args.precision == "mixed" else None),
        "stages_ms": {k: round(st[k], 4) for k in ("ms_bin", "ms_assemble", "ms_solve", "ms_pair_screen",
                                                   "ms_pair_eval", "ms_adjoint")},
        "mg": {"levels": st["mg_levels"], "iterations": st["mg_iterations"], "refine_steps": st["refine_steps"],
               "rel_residual": st["mg_rel_residual"], "adj_iterations": st["adj_iterations"]},
        "roofline": roof,
        "roofline_pair": roof_pair,
        "e2e": {"value": round(e2e_value, 1), "unit": "particles/s", "h2d_bytes_per_step": N * 32,
                "d2h_bytes_per_step": N * 8 + N * 24 + 8},
        "gpu_launches": int(round(main["launches"])),
        "clocks": main["clocks"],
    }
    if args.large and ws == 1:
        # the full-size workloads of the other configurations, mixed with forces (not the headline)
        line["workloads"] = {nm: large_workload(nm, st_, 3, flush, dev, torch, peaks)
                             for nm, st_ in (("water1m", 20), ("blobs4m", 10))}
        for kind in ("dirichlet", "neumann"):
            line["workloads"]["box_%s_nacl32" % kind] = box_workload(kind, 10, 3, flush, dev, torch)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def oracle_step(d):
    from oracle import fep3m as ofe
    f = ofe.forward(d["pos"], d["Q"], d["L"], d["n_el"], want_grad=True)
    dx, _, _ = ofe.vjp(f, d["Q"])
    return f["U"], dx


ONE_THREAD = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def cpu_baseline():
    """The CPU oracle, as it stands, on the full workload (one step: Phi, U and forces), on all host cores,
    and again in a child process whose BLAS and OpenMP pools are limited to one thread."""
    from oracle import tables
    from paper_1503_08509_gb300 import workloads
    d = workloads.workload(WORKLOAD)
    tables.kept_table()                     # create-time table, not timed (as on the GPU)
    t0 = time.perf_counter()
    oracle_step(d)
    dt = time.perf_counter() - t0
    res = {"value": round(len(d["Q"]) / dt, 1), "unit": "particles/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "full workload, one step (numpy/scipy FP64; BLAS threads = all cores)",
           "seconds": round(dt, 2)}
    env = dict(os.environ, **{k: "1" for k in ONE_THREAD})
    code = ("import sys, time; sys.path.insert(0, %r); import bench; from oracle import tables; "
            "from paper_1503_08509_gb300 import workloads; d = workloads.workload(bench.WORKLOAD); "
            "tables.kept_table(); t0 = time.perf_counter(); bench.oracle_step(d); "
            "print(time.perf_counter() - t0)" % ROOT)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        dt1 = float(r.stdout.strip().splitlines()[-1])
        res["one_thread"] = {"value": round(len(d["Q"]) / dt1, 1), "unit": "particles/s", "cores": 1,
                             "seconds": round(dt1, 2),
                             "sample": "the same step in a child process with %s = 1" % "/".join(ONE_THREAD)}
    except Exception as exc:   # reported, not fatal: the all-core figure stands
        res["one_thread"] = {"error": str(exc)[:200]}
    return res


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return
    from oracle import tables
    from paper_1503_08509_gb300 import workloads
    d = workloads.workload(WORKLOAD)
    N = len(d["Q"])
    tables.kept_table()
    for _ in range(min(args.warmup, 1)):
        oracle_step(d)
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        oracle_step(d)
        times.append(time.perf_counter() - t0)
    value = N * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "particles/s",
            "n_gpus": ws, "steps": len(times), "warmup": min(args.warmup, 1),
            "ms_per_step": round(1e3 * sum(times) / len(times), 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "jittered rock salt 32^3 = 32768 ions, periodic 32^3 hex mesh, q=1, 7^3 block",
                       "step": "oracle forward (Phi, U) + adjoint forces"},
            "cpu_baseline": {"value": round(value, 1), "unit": "particles/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "full workload per step; steps capped at 3"},
            "e2e": {"value": round(value, 1), "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
