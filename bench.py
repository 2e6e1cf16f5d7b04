"""Benchmark: geometric-multigrid V-cycle solves of 2D generalized Stokes on one GB300.

Workload (one "step"): the sigma/nu sweep {1e-4, 1e-2, 1, 1e2, 1e4} (nu = 1) of the
2D generalized Stokes problem on the unit square, streamfunction degree p = 2 and 3,
256 x 256 fine elements, 7 grids (coarsest 4 x 4), V(2,2) multiplicative Schwarz, FP64,
forcing from a seeded Gaussian random field (squared-exponential kernel, length 0.1),
zero initial guess, solved to a 1e-8 relative residual: 10 solves per step.

Metric: MDOF/s per V-cycle = sum over solves of (DOFs x V-cycles) / time / 1e6, for the
plain FP64 GPU multigrid (the line's value), with the solve time to 1e-8 also reported; the
same sweep solved by FP32 V-cycles inside FP64 iterative refinement is reported beside it
(same tolerance, its own time and speed-up over FP64).  Inputs are resident in HBM when the timed region
starts; L2 is flushed (a 512 MB write) before every timed step, outside its events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
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

METRIC = "solve time to 1e-8 rel. residual & MDOF/s per V-cycle vs plain FP64 GPU MG"
SIGMAS = [1e-4, 1e-2, 1.0, 1e2, 1e4]
DEGREES = [2, 3]
N_FINE, N_LEVELS, RTOL, MAXC = 256, 7, 1e-8, 60
SEED = 1706
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def workload_config():
    return {"workload": "2D generalized Stokes, unit square, div-conforming B-splines p=2,3, "
                        "256x256 fine elements, 7 levels, sigma/nu in {1e-4,1e-2,1,1e2,1e4}, "
                        "GRF forcing (SE kernel, length 0.1), V(2,2) multiplicative Schwarz, "
                        "FP64, zero initial guess, to 1e-8 relative residual",
            "n_fine": N_FINE, "n_levels": N_LEVELS, "degrees": DEGREES, "sigma_over_nu": SIGMAS,
            "solves_per_step": len(SIGMAS) * len(DEGREES), "l2": "flushed before each step (512 MB write)"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


def max_over_ranks(seconds, device, world):
    """The job's time: the maximum of the ranks' timed regions (replicas run the same sweep;
    value = all ranks' work / this time)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons during the timed region."""

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_fma_peak(dev, stream, fp64=True, repeats=5):
    """Measured FMA throughput of this GPU (TFLOP/s): igamg_probe_fma, 8 independent
    multiply-add chains per thread, 8 blocks of 256 threads per SM, best of `repeats`
    CUDA-event timings on `stream` after one warm-up launch."""
    import ctypes

    import torch

    from paper_1705_09282_gb300 import _lib
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = sms * 8, (4096 if fp64 else 65536)
    out = torch.empty(blocks * 256, dtype=torch.float64 if fp64 else torch.float32, device=dev)
    flops = ctypes.c_double()
    st = ctypes.c_void_p(stream.cuda_stream)
    best = None
    for k in range(repeats + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rc = _lib.lib().igamg_probe_fma(1 if fp64 else 0, blocks, iters, ctypes.c_void_p(out.data_ptr()), st,
                                        ctypes.byref(flops))
        e1.record(stream)
        torch.cuda.synchronize()
        assert rc == 0, rc
        t = e0.elapsed_time(e1) / 1e3
        if k > 0:
            best = t if best is None else min(best, t)
    return flops.value / best / 1e12


def launches_per_solve(p, cycles, mixed=False):
    """Kernels of ours in one igamg_solve (an upper estimate: a fused coarse end, when the
    autotuner picks one, replaces several of them by one): per V-cycle, per smoothed level
    two pipelined sweep launches (pre and post) + residual (2) + restriction +
    prolongation; coarse solve; the fine residual norm (2).  The FP32 mode adds the
    down-cast, the streamfunction integration and the curl update per cycle.  Plus the
    initial residual (2) and the final divergence check."""
    per_cycle = (N_LEVELS - 1) * (2 + 2 + 1 + 1) + 1 + 2 + (3 if mixed else 0)
    return 2 + cycles * per_cycle + 1


def run_ours(args):
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IGAMG_FGMRES_FP32, IGAMG_FGMRES_FP64, IGAMG_FP32_IR
    from paper_1705_09282_gb300.solver import Solver, solve_batch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    stream = torch.cuda.current_stream(dev)
    problems = []
    for p in DEGREES:
        f_host = inputs.grf_forcing(p, N_FINE, seed=SEED)
        f_dev = torch.tensor(f_host, device=dev)
        for s in SIGMAS:
            S = Solver(p, N_FINE, N_LEVELS, s, 1.0, nu1=2, nu2=2, device=dev, stream=stream)
            S32 = Solver(p, N_FINE, N_LEVELS, s, 1.0, nu1=2, nu2=2, device=dev, stream=stream,
                         precision=IGAMG_FP32_IR)
            os.environ["IGAMG_BF16_OPERANDS"] = "1"     # the BF16-operand variant of the same
            S16 = Solver(p, N_FINE, N_LEVELS, s, 1.0, nu1=2, nu2=2, device=dev, stream=stream,
                         precision=IGAMG_FP32_IR)
            del os.environ["IGAMG_BF16_OPERANDS"]
            F = S.load_vector(f_dev)
            problems.append({"p": p, "sigma": s, "S": S, "S32": S32, "S16": S16, "F": F, "U": S.empty(),
                             "f_host": f_host, "ndof": S.ndof()})
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(key="S"):
        """The whole sweep: all solves side by side through igamg_solve_batch."""
        for pr in problems:
            pr["U"].zero_()
        reps = solve_batch([pr[key] for pr in problems], [pr["U"] for pr in problems],
                           [pr["F"] for pr in problems], rtol=RTOL, max_cycles=MAXC)
        tot_dof_cycles, cycles, worst = 0, [], 0.0
        for pr, rep in zip(problems, reps):
            if key == "S16" and not rep["converged"]:      # reported, not fatal: an experiment
                cycles.append(-1)
                continue
            assert rep["converged"], (pr["p"], pr["sigma"], key, rep)
            tot_dof_cycles += pr["ndof"] * rep["cycles"]
            cycles.append(rep["cycles"])
            worst = max(worst, rep["div_inf"])
        return tot_dof_cycles, cycles, worst

    def single_solve_ms(key):
        """Latency of one solve alone (the first problem), for context."""
        pr = problems[0]
        pr["U"].zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = pr[key].solve(pr["U"], pr["F"], rtol=RTOL, max_cycles=MAXC, history=False)
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0), rep["cycles"]

    def timed(key, steps):
        ms, dofcyc, cyc, worst = [], 0, None, 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            dc, cyc, w = step(key)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            dofcyc += dc
            worst = max(worst, w)
        return ms, dofcyc, cyc, worst

    for _ in range(args.warmup):
        step("S")
        step("S32")
        step("S16")
    torch.cuda.synchronize()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    torch.cuda.nvtx.range_push("timed_fp64")     # lets a profiler select the timed FP64 steps
    ms_steps, dofcyc, cyc_list, div64 = timed("S", args.steps)
    torch.cuda.nvtx.range_pop()
    ms32, dofcyc32, cyc32, div32 = timed("S32", args.steps)
    ms16, dofcyc16, cyc16, div16 = timed("S16", args.steps)
    clocks = clk.stop()
    lat64, lat64_cyc = single_solve_ms("S")
    lat32, lat32_cyc = single_solve_ms("S32")
    # the Krylov wrapper on the same single solve (FGMRES(20) in FP64, V-cycle preconditioner)
    krylov = {}
    pr0 = problems[0]
    for name, prec in (("fgmres_fp64", IGAMG_FGMRES_FP64), ("fgmres_fp32", IGAMG_FGMRES_FP32)):
        SK = Solver(pr0["p"], N_FINE, N_LEVELS, pr0["sigma"], 1.0, nu1=2, nu2=2, device=dev, stream=stream,
                    precision=prec, restart=20)
        for _ in range(2):
            pr0["U"].zero_()
            rk = SK.solve(pr0["U"], pr0["F"], rtol=RTOL, max_cycles=MAXC, history=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr0["U"].zero_()
        rk = SK.solve(pr0["U"], pr0["F"], rtol=RTOL, max_cycles=MAXC, history=False)
        torch.cuda.synchronize()
        krylov[name] = {"single_solve_ms": 1e3 * (time.perf_counter() - t0), "vcycles": rk["cycles"],
                        "converged": rk["converged"], "rel_residual": rk["rel_residual"], "div_inf": rk["div_inf"]}
        SK.close()
    t_total = max_over_ranks(sum(ms_steps) / 1e3, dev, world)
    value = world * dofcyc / t_total / 1e6
    solves = len(problems)
    solve_ms = 1e3 * t_total / (args.steps * solves)
    t32 = sum(ms32) / 1e3
    mixed = {"precision": "FP32 V-cycles (FP32 smoother, operator, transfers, coarse solve) inside FP64 "
                          "iterative refinement; FP64 outer residual; velocity update = FP64 curl of a streamfunction",
             "value": world * dofcyc32 / t32 / 1e6, "unit": "MDOF/s per V-cycle",
             "solve_ms_to_1e-8": 1e3 * t32 / (args.steps * solves),
             "speedup_vs_fp64_solve_time": t_total / t32,
             "single_solve_ms": lat32, "single_solve_case": f"p=2, sigma=1e-4, {lat32_cyc} cycles",
             "cycles": {f"p{pr['p']}_sigma{pr['sigma']:g}": c for pr, c in zip(problems, cyc32)},
             "max_div_inf": div32}
    t16 = sum(ms16) / 1e3
    bf16 = {"precision": "as mixed_fp32_ir, with the operator's stencil records and the patch solves' local "
                         "inverses rounded to bfloat16 (FP32 accumulation; transfers and the coarsest solve FP32)",
            "value": world * dofcyc16 / t16 / 1e6, "unit": "MDOF/s per V-cycle",
            "solve_ms_to_1e-8": 1e3 * t16 / (args.steps * solves),
            "speedup_vs_fp64_solve_time": t_total / t16,
            "cycles": {f"p{pr['p']}_sigma{pr['sigma']:g}": c for pr, c in zip(problems, cyc16)},
            "max_div_inf": div16,
            "storage_note": "operands rounded to bf16 values and kept in FP32 words: the arithmetic of bf16 "
                            "operands, not their storage (the sweep is latency-bound, see the FP32 roofline)"}

    # ---- dominant kernel: the finest level's multiplicative sweep ------------------------
    # nu = 2 sweeps (all colours) of the finest level, as in every V-cycle's pre- and
    # post-smoothing, in the form the autotuner chose for that level, captured into a CUDA
    # graph (the way solves run it) on a side stream and replayed 10 times between CUDA
    # events on that stream; the average per colour launch (or per pipelined launch) is the
    # kernel's launch duration.
    pk, pk_src = peaks()
    pr0 = problems[0]
    p0 = pr0["p"]
    side = torch.cuda.Stream(dev)
    Sr = Solver(p0, N_FINE, N_LEVELS, pr0["sigma"], 1.0, nu1=2, nu2=2, device=dev, stream=side,
                precision=IGAMG_FP32_IR)
    sz = Sr.sizes()
    form = Sr.level_form()
    with torch.cuda.stream(side):
        Ur = torch.zeros(sz.n_total, dtype=torch.float64, device=dev)
        Fr = pr0["F"].clone()
        Ur32 = torch.zeros(sz.n_total, dtype=torch.float32, device=dev)
        Fr32 = Fr.to(torch.float32)
    side.synchronize()
    # algorithmic FP64 flops per patch and sweep: its 8 residual rows (2 flops per stencil
    # coefficient: u_x, u_y rows (4p+1)(2p-1), p rows 4p(2p-1)+1), the 8x8 local inverse
    # (2 x 64) and 16 adds
    rx, rp = (4 * p0 + 1) * (2 * p0 - 1), 4 * p0 * (2 * p0 - 1) + 1
    flops_patch = 2 * (4 * rx + 4 * rp) + 2 * 64 + 16
    sweeps_per_replay, replays = 2, 10

    def graph_sweep_s(smooth, U, F):
        for _ in range(2):
            with torch.cuda.stream(side):
                smooth(U, F, sweeps=sweeps_per_replay)
        side.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            smooth(U, F, sweeps=sweeps_per_replay)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):           # replay() launches on the current stream
            g.replay()
            e0.record(side)
            for _ in range(replays):
                g.replay()
            e1.record(side)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / replays

    t_sweeps = graph_sweep_s(Sr.smooth, Ur, Fr)
    t_sweeps32 = graph_sweep_s(Sr.smooth32, Ur32, Fr32)
    launches_per_replay = 1 if form["tiles"] else sweeps_per_replay * sz.n_colours
    launch_s = t_sweeps / launches_per_replay
    flops_replay = sz.n_patches * sweeps_per_replay * flops_patch
    achieved = flops_replay / t_sweeps / 1e12
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp64_derived = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12    # 152 SMs x 2 DFMA/clk x 2 flops
    fp64_peak = measured_fma_peak(dev, stream, fp64=True)
    fp32_peak = measured_fma_peak(dev, stream, fp64=False)
    # algorithmic bytes per sweep: U read and written once, F read once, the patch DOF lists
    # (8 int32 per patch) and class ids read once
    bytes_replay = sweeps_per_replay * (3 * 8 * sz.n_total + sz.n_patches * (8 + 1) * 4)
    if form["tiles"]:
        kname = (f"k_sweep_tiles<{p0},double> (pipelined: {form['tiles']} tiles of {form['threads']} threads; "
                 f"one launch = 2 sweeps x {sz.n_colours} colours)")
    else:
        kname = (f"k_mult_colour<{p0},double,{form['lanes']},{form['chains']}> (one colour of the finest level "
                 f"{N_FINE}^2, {form['lanes']} lane(s) per patch row, {form['chains']} multiply-add chains, "
                 f"{form['threads']}-thread blocks; autotuned form)")
    # DRAM bytes (read + write) per launch from the ncu captures of this kernel in the same form
    # (colours 0 and 1 of the 256^2 finest level, mean of the two launches), for the forms
    # captured; none for another form
    captured = {(1, 64, 0, 4): 3.21e6, (1, 64, 0, 2): 3.208e6}
    traffic = captured.get((form["lanes"], form["threads"], form["tiles"], form["chains"])) if p0 == 2 else None
    roofline = {"kernel": kname, "bound": "alu",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s (FP64)", "frac": achieved / fp64_peak,
                "traffic": traffic, "traffic_unit": "bytes per launch",
                "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum of this kernel in this form, one ncu "
                                 "capture of colours 0 and 1 (cold L2): profiles/k_mult_colour_p2_fp64_256x256.md"
                                 if traffic else "this form has no ncu capture"),
                "peak_source": "measured: igamg_probe_fma, FP64 FMA chains on every SM, best of 5 (CUDA events)",
                "peak_derived": fp64_derived, "fp32_peak_measured": fp32_peak,
                "avg_launch_us": launch_s * 1e6, "launches_timed": launches_per_replay * replays,
                "flops_per_launch": flops_replay / launches_per_replay,
                "algorithmic_bytes_per_launch": bytes_replay / launches_per_replay,
                "achieved_gbs_algorithmic": bytes_replay / t_sweeps / 1e9,
                "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_source": pk_src, "form": form,
                "timing": "2 sweeps captured in a CUDA graph on a side stream, 10 replays between CUDA events",
                "working_set_note": "finest-level vectors (1.6 MB) stay in L2; the kernel is FP64-issue bound"}
    # the FP32 inner smoother of the mixed mode, same launches
    bytes32 = sweeps_per_replay * (3 * 4 * sz.n_total + sz.n_patches * (8 + 1) * 4)
    roofline32 = {"kernel": kname.replace(",double", ",float").replace(f",{form['chains']}>", ",4>").replace(
                      f"{form['chains']} multiply-add chains", "4 multiply-add chains"), "bound": "latency",
                  "avg_launch_us": t_sweeps32 / launches_per_replay * 1e6,
                  "achieved_tflops": flops_replay / t_sweeps32 / 1e12, "fp32_peak_measured": fp32_peak,
                  "frac_fp32_peak": flops_replay / t_sweeps32 / 1e12 / fp32_peak,
                  "algorithmic_bytes_per_launch": bytes32 / launches_per_replay,
                  "achieved_gbs_algorithmic": bytes32 / t_sweeps32 / 1e9, "hbm_peak_gbs": pk["hbm_gbs"],
                  "frac_hbm": bytes32 / t_sweeps32 / 1e9 / pk["hbm_gbs"],
                  "speedup_vs_fp64": t_sweeps / t_sweeps32}
    mixed["roofline"] = roofline32
    Sr.close()

    # ---- end to end through the host-buffer C-ABI call --------------------------------
    # The same 10 solves, each through igamg_solve_host (forcing from pinned host memory in,
    # solution back out, both copies inside the call), side by side like the device-resident
    # sweep: one handle per solve on its own stream, the calls from 10 host threads.
    from concurrent.futures import ThreadPoolExecutor
    legs = []
    for pr in problems:
        st = torch.cuda.Stream(dev)
        Sh = Solver(pr["p"], N_FINE, N_LEVELS, pr["sigma"], 1.0, nu1=2, nu2=2, device=dev, stream=st)
        legs.append({"S": Sh, "f": torch.tensor(pr["f_host"]).pin_memory(),
                     "u": torch.zeros(pr["ndof"], dtype=torch.float64).pin_memory(), "ndof": pr["ndof"]})

    def host_solve(leg):
        leg["u"].zero_()
        return leg["S"].solve_host(leg["f"].numpy(), leg["u"].numpy(), rtol=RTOL, max_cycles=MAXC)

    pool = ThreadPoolExecutor(max_workers=len(legs))
    list(pool.map(host_solve, legs))                  # warm-up (graph capture of the host workspaces)
    h2d = d2h = 0
    e2e_dofcyc = 0
    nrep = max(1, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(nrep):
        reps = list(pool.map(host_solve, legs))
        for leg, rep in zip(legs, reps):
            e2e_dofcyc += leg["ndof"] * rep["cycles"]
            h2d += leg["f"].numel() * 8 + leg["u"].numel() * 8
            d2h += leg["u"].numel() * 8
    t_e2e = time.perf_counter() - t0
    pool.shutdown()
    e2e = {"value": world * e2e_dofcyc / t_e2e / 1e6, "unit": "MDOF/s per V-cycle",
           "h2d_bytes_per_step": h2d // nrep, "d2h_bytes_per_step": d2h // nrep,
           "solve_ms": 1e3 * t_e2e / (nrep * solves),
           "note": "10 host-buffer solves side by side (one handle and stream each, 10 host threads)"}
    for leg in legs:
        leg["S"].close()

    line = {"metric": METRIC, "value": value, "unit": "MDOF/s per V-cycle", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian random field forcing)", "config": workload_config(),
            "solve_ms_to_1e-8": solve_ms,
            "solve_ms_note": "sweep time / solves, the 10 solves running side by side (igamg_solve_batch)",
            "single_solve_ms": lat64, "single_solve_case": f"p=2, sigma=1e-4, {lat64_cyc} cycles, alone",
            "cycles": {f"p{pr['p']}_sigma{pr['sigma']:g}": c for pr, c in zip(problems, cyc_list)},
            "roofline": roofline, "e2e": e2e, "clocks": clocks, "mixed_fp32_ir": mixed, "mixed_bf16_operands_ir": bf16,
            "krylov_single_solve": krylov,
            "max_div_inf": div64,
            "gpu_launches": (sum(launches_per_solve(pr["p"], c) for pr, c in zip(problems, cyc_list))
                             + sum(launches_per_solve(pr["p"], c, mixed=True) for pr, c in zip(problems, cyc32))
            + sum(launches_per_solve(pr["p"], c, mixed=True) for pr, c in zip(problems, cyc16))) * args.steps}
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(line), flush=True)
    for pr in problems:
        pr["S"].close()
        pr["S32"].close()
        pr["S16"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_vcycle_sample(n_cycles=1):
    """The oracle as it stands on the host: one V-cycle of the p=2, sigma=nu=1 solve
    at 256 x 256 (set-up not timed)."""
    import numpy as np

    from oracle import stokes2d as o2
    from paper_1705_09282_gb300 import inputs
    H = o2.Hierarchy(2, N_FINE, N_LEVELS, 1.0, 1.0, nu1=2, nu2=2)
    F = H.fine.load_vector(inputs.grf_forcing(2, N_FINE, seed=SEED))
    U = np.zeros_like(F)
    return H, U, F


def cpu_baseline_sample():
    H, U, F = _oracle_vcycle_sample()
    t0 = time.perf_counter()
    H.vcycle(U, F)
    dt = time.perf_counter() - t0
    return {"value": len(F) / dt / 1e6, "unit": "MDOF/s per V-cycle", "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "one V-cycle of the p=2, sigma=nu=1 solve at 256x256 (7 grids, V(2,2)), "
                      "single-threaded numpy/scipy, set-up not timed", "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    H, U, F = _oracle_vcycle_sample()
    for _ in range(args.warmup):
        H.vcycle(U, F)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.vcycle(U, F)
    dt = time.perf_counter() - t0
    v = args.steps * len(F) / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": "MDOF/s per V-cycle", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian random field forcing)", "config": workload_config(),
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "MDOF/s per V-cycle", "kind": "oracle", "cores": 1,
                             "host_cores": os.cpu_count(),
                             "sample": "each step one V-cycle of the p=2, sigma=nu=1 solve at 256x256"},
            "e2e": {"value": v, "unit": "MDOF/s per V-cycle", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(spec):
    """Untimed workload for profilers: two solves of one case of the sweep.
    spec = "p<degree>-<fp64|mixed>[-sigma<value>]", e.g. "p2-fp64", "cube-p2-<fp64|mixed>" (one
    solve of the 64^3 cube), "oseen-<fp64|mixed>" (one solve of the 512^2 Oseen problem),
    "batch128" (two lockstep batches of 24 solves of 128^2) or "nn" (network inference)."""
    import numpy as np
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR, IGAMG_FP64
    from paper_1705_09282_gb300.solver import Solver
    parts = spec.split("-")
    if parts[0] == "nn":
        # warm-start network inference: 16 inputs of 130 x 130 (the 128^2 problems' grid),
        # dilations (1, 2, 4, 8), twice
        from paper_1705_09282_gb300.warmstart import Network
        net = Network(seed=1)
        x = torch.randn((16, 3, 130, 130), dtype=torch.float32, device="cuda")
        for _ in range(2):
            y = net.forward(x)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": spec, "out_abs_max": float(y.abs().max())}))
        return
    if parts[0] == "batch128":
        # 24 solves of 128^2 (p = 2, 6 grids, sigma/nu spread over [1e-2, 1e4]) in one lockstep group
        from paper_1705_09282_gb300.solver import solve_batch
        solvers, Us, Fs = [], [], []
        for j, sig in enumerate(np.logspace(-2, 4, 24)):
            S = Solver(2, 128, 6, float(sig), 1.0)
            Fs.append(S.load_vector(torch.tensor(inputs.grf_forcing(2, 128, seed=1709 + j), device="cuda")))
            Us.append(S.empty())
            solvers.append(S)
        for _ in range(2):
            for U in Us:
                U.zero_()
            reps = solve_batch(solvers, Us, Fs, rtol=RTOL, max_cycles=MAXC)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": spec, "cycles": [r["cycles"] for r in reps]}))
        return
    if parts[0] == "oseen":
        prec = IGAMG_FP32_IR if parts[1] == "mixed" else IGAMG_FP64
        S = Solver(2, 512, 8, 1.0, 1e-2, beta=inputs.oseen_advection(2, 512, 0.5), precision=prec)
        F = S.load_vector(torch.tensor(inputs.grf_forcing(2, 512, seed=1707), device="cuda"))
        U = S.empty()
        rep = S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": spec, "cycles": rep["cycles"], "rel_residual": rep["rel_residual"]}))
        return
    if parts[0] == "cube":
        prec = IGAMG_FP32_IR if parts[2] == "mixed" else IGAMG_FP64
        S = Solver(int(parts[1][1:]), 64, 5, 1.0, 1.0, nu1=2, nu2=2, precision=prec, dim=3)
        F = S.load_vector(torch.tensor(inputs.manufactured_forcing_3d(S.p, 64, 1.0, 1.0), device="cuda"))
        U = S.empty()
        rep = S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": spec, "cycles": rep["cycles"], "rel_residual": rep["rel_residual"]}))
        return
    p = int(parts[0][1:])
    prec = IGAMG_FP32_IR if parts[1] == "mixed" else IGAMG_FP64
    sigma = float(parts[2][5:]) if len(parts) > 2 else 1.0
    S = Solver(p, N_FINE, N_LEVELS, sigma, 1.0, nu1=2, nu2=2, precision=prec)
    F = S.load_vector(torch.tensor(inputs.grf_forcing(p, N_FINE, seed=SEED), device="cuda"))
    U = S.empty()
    for _ in range(2):
        U.zero_()
        rep = S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": spec, "cycles": rep["cycles"], "rel_residual": rep["rel_residual"]}))


def _timed(fn, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def run_oseen(args):
    """Generalized Oseen, 512 x 512, 8 grids, p = 2, nu = 1e-2, sigma = 1, advection the curl
    of sin^2(pi x) sin^2(pi y) scaled to max |beta| = 0.5 (Re = 50 < Da = 100), GRF forcing:
    FP64 and FP32-in-FP64 solves to 1e-8; the finest residual in both operator forms (per-row
    records, matrix-free advection) with their rooflines."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR, IGAMG_FP64, IgamgError
    from paper_1705_09282_gb300.solver import Solver
    p, n, L, sigma, nu = 2, 512, 8, 1.0, 1e-2
    beta = inputs.oseen_advection(p, n, 0.5)
    f = torch.tensor(inputs.grf_forcing(p, n, seed=1707), device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec in (("fp64", IGAMG_FP64), ("mixed", IGAMG_FP32_IR)):
        t0 = time.perf_counter()
        try:
            S = Solver(p, n, L, sigma, nu, beta=beta, precision=prec)
        except IgamgError as e:
            out[name] = {"error": str(e)}
            continue
        setup = time.perf_counter() - t0
        F = S.load_vector(f)
        U = S.empty()
        for _ in range(args.warmup):
            U.zero_()
            S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
        ts, cyc = [], None
        for _ in range(args.steps):
            U.zero_()
            dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False), stream)
            assert rep["converged"], rep
            ts.append(dt)
            cyc, div = rep["cycles"], rep["div_inf"]
        t = sum(ts) / len(ts)
        # the FP64 colour kernel on the finest level, timed alone
        sz = S.sizes()
        sweeps = 10
        dt_sm, _ = _timed(lambda: S.smooth(U, F, sweeps=sweeps), stream)
        colour_us = 1e6 * dt_sm / (sweeps * sz.n_colours)
        # the finest residual (operator apply) in both forms: per-row records (Stokes part and
        # advection stored per row, streamed from HBM) and the advection matrix-free (element by
        # element at the (p+2)^2 Gauss points, sum-factorised; Stokes part from class stencils)
        ntot, G = sz.n_total, p + 2
        nG = n * G
        RU = (2 * p + 1) * (2 * p - 1) + 2 * p * (2 * p - 1) + 1   # padded row record (2 boxes + lambda)
        Q = p - 1
        fma_ux = (2 * (Q + 1) * G * (p + 1) + 2 * G * G * (Q + 1) + 2 * G * G + G * (p + 1) * G
                  + G * (p + 1) * (Q + 1))
        fma_uy = (2 * (p + 1) * G * (Q + 1) + 2 * G * G * (p + 1) + 2 * G * G + G * (Q + 1) * G
                  + G * (Q + 1) * (p + 1))
        forms = S.residual_form()
        res = {}
        for prec_name, w in (("fp64", 8), ("fp32", 4)):
            if forms[prec_name] < 1:
                continue
            if prec_name == "fp64":
                Ur, Fr, Rr = U, F, S.empty()
                call = lambda: S.residual(Ur, Fr, out=Rr)        # noqa: E731
            else:
                Ur = torch.randn(ntot, dtype=torch.float32, device="cuda")
                Fr = torch.randn(ntot, dtype=torch.float32, device="cuda")
                Rr = torch.empty_like(Fr)
                call = lambda: S.residual32(Ur, Fr, out=Rr)      # noqa: E731
            entry = {"chosen": "matrix_free" if forms[prec_name] == 2 else "records"}
            for code, fname in ((1, "records"), (2, "matrix_free")):
                S.set_residual_form(**{prec_name: code})
                call()
                reps_r = 50
                dt_r, _ = _timed(lambda: [call() for _ in range(reps_r)], stream)
                us = 1e6 * dt_r / reps_r
                if code == 1:
                    nbytes = (ntot - 1) * (RU + 3) * w                    # records + U, F, R once
                    flops = 2.0 * (ntot - 1) * RU
                else:
                    nbytes = (3 * ntot + 2 * nG * nG) * w                 # U, F, R + w*beta at the Gauss points
                    flops = 2.0 * (n * n * (fma_ux + fma_uy) + (ntot - 1) * RU)
                entry[fname] = {"us_per_launch": us, "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / us / 1e3,
                                "algorithmic_flops": flops, "achieved_tflops": flops / us / 1e6}
            S.set_residual_form(**{prec_name: forms[prec_name]})
            res[prec_name] = entry
        # colour: per 8-DOF patch 8 records, its own 8x8 inverse, dof ids, class id, F and U rows
        patches_colour = sz.n_patches / sz.n_colours
        col_bytes = patches_colour * (8 * RU * 8 + 64 * 8 + 8 * 4 + 4 + 3 * 8 * 8)
        out[name] = {"solve_ms": 1e3 * t, "cycles": cyc, "mdof_per_s_per_cycle": S.ndof() * cyc / t / 1e6,
                     "div_inf": div, "setup_s": setup, "fp64_colour_launch_us": colour_us,
                     "residual_forms": res,
                     "colour_hbm": {"bytes": col_bytes, "achieved_gbs": col_bytes / colour_us / 1e3}}
        S.close()
    pk, src = peaks()
    dev = torch.device("cuda")
    fma = {"fp64": measured_fma_peak(dev, stream, True), "fp32": measured_fma_peak(dev, stream, False)}
    for v in out.values():
        if "error" in v:
            continue
        v["colour_hbm"]["peak_gbs"] = pk["hbm_gbs"]
        v["colour_hbm"]["frac"] = v["colour_hbm"]["achieved_gbs"] / pk["hbm_gbs"]
        for prec_name, entry in v["residual_forms"].items():
            for fname in ("records", "matrix_free"):
                e = entry[fname]
                e["frac_hbm"] = e["achieved_gbs"] / pk["hbm_gbs"]
                e["frac_fma_peak"] = e["achieved_tflops"] / fma[prec_name]
            entry["fma_peak_tflops_measured"] = fma[prec_name]
    line = {"metric": "Oseen solve time to 1e-8 rel. residual (2D, 512^2)", "workload": "oseen",
            "config": {"workload": "2D generalized Oseen, unit square, p=2, 512x512, 8 levels, nu=1e-2, sigma=1, "
                                   "max|beta|=0.5 (Re=50, Da=100), GRF forcing seed 1707, V(2,2) multiplicative",
                       "ndof": None}, "results": out, "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_source": src}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The 1024-solve batch: independent 2D generalized Stokes solves of sizes 64/96/128
    (round-robin), sigma/nu log-uniform in [1e-2, 1e4], GRF forcing, side by side; zero
    initial guess versus the learned warm start (network trained on separate problems
    solved by the same multigrid), both to the absolute residual 1e-8 ||F||."""
    import numpy as np
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300 import warmstart as ws
    p = 2
    count = args.batch_count
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    probs = [ws.Problem(p, n, ws.levels_for(n), s, nu, seed) for (n, s, nu, seed) in inputs.batch_problems(count, 1709)]
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    train = [ws.Problem(p, n, ws.levels_for(n), s, nu, seed)
             for (n, s, nu, seed) in inputs.batch_problems(args.train_count, 50000)]
    grids = ws.targets(train)
    net = ws.Network(seed=1)
    losses = ws.train(net, train, grids, steps=args.train_steps, batch=16, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    atol = [1e-8 * float(torch.linalg.norm(pr.F)) for pr in probs]
    ndof = np.array([pr.solver.ndof() for pr in probs])

    def cold():
        for pr in probs:
            pr.U.zero_()
        return ws.solve_batch_abs([pr.solver for pr in probs], [pr.U for pr in probs], [pr.F for pr in probs], atol, MAXC)

    def warm(scaled=False):
        ws.predict_guesses(net, probs, scaled=scaled)
        return ws.solve_batch_abs([pr.solver for pr in probs], [pr.U for pr in probs], [pr.F for pr in probs], atol, MAXC)

    cold()
    warm()
    warm(True)

    def infer_all():
        for pr in probs:
            net.forward(pr.x.unsqueeze(0).contiguous())

    infer = {}
    for mode in ("1", "0"):                  # tensor-core (tcgen05) or SIMT 32 -> 32 layers
        os.environ["IGAMG_NN_TC"] = mode
        infer_all()
        infer["tcgen05" if mode == "1" else "simt"] = _timed(infer_all, stream)[0]
    del os.environ["IGAMG_NN_TC"]
    tc, rc = _timed(cold, stream)
    tw, rw = _timed(warm, stream)
    ts, rs = _timed(lambda: warm(True), stream)
    cc = np.array([r["cycles"] for r in rc])
    cw = np.array([r["cycles"] for r in rw])
    cs = np.array([r["cycles"] for r in rs])
    line = {"metric": "batched solve time to 1e-8 ||F|| and MDOF/s per V-cycle (1024 solves of 64^2..128^2)", "workload": "batch",
            "config": {"solves": count, "sizes": [64, 96, 128], "p": p, "sigma_over_nu": "log-uniform [1e-2, 1e4]",
                       "train_problems": args.train_count, "train_steps": args.train_steps},
            "zero_guess": {"seconds": tc, "mean_cycles": float(cc.mean()), "mdof_per_s_per_cycle": float((ndof * cc).sum() / tc / 1e6)},
            "warm_start": {"seconds": tw, "mean_cycles": float(cw.mean()), "mdof_per_s_per_cycle": float((ndof * cw).sum() / tw / 1e6),
                           "includes": "network inference and curl of the predicted streamfunction for every solve",
                           "cycles_saved_total": int(cc.sum() - cw.sum()), "worse_count": int((cw > cc).sum())},
            "warm_start_scaled": {"seconds": ts, "mean_cycles": float(cs.mean()),
                                  "mdof_per_s_per_cycle": float((ndof * cs).sum() / ts / 1e6),
                                  "includes": "as warm_start, plus the residual-minimising scaling of the two "
                                              "predicted fields (igamg_warm_start_minres) for every solve",
                                  "cycles_saved_total": int(cc.sum() - cs.sum()), "worse_count": int((cs > cc).sum()),
                                  "max_res0_over_normF": max(r["res0"] / (a / 1e-8) for r, a in zip(rs, atol))},
            "inference_s_all_solves": infer,
            "max_div_inf": max(r["div_inf"] for r in rw + rs), "setup_s": t_setup, "train_s": t_train,
            "train_loss_first_last": [float(np.mean(losses[:5])), float(np.mean(losses[-20:]))]}
    print(json.dumps(line), flush=True)


def run_cube(args):
    """3D generalized Stokes on the unit cube: p = 2, 64^3 elements, 5 grids, sigma/nu in
    {1, 1e3}, the cube's manufactured forcing (Sec. 6.3), V(2,2) multiplicative smoother over
    the vector-potential supports; FP64 and FP32-in-FP64 solves from zero to 1e-8."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR, IGAMG_FP64
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 64, 5
    stream = torch.cuda.current_stream()
    out = {}
    for sigma in (1.0, 1e3):
        f = torch.tensor(inputs.manufactured_forcing_3d(p, n, sigma, 1.0), device="cuda")
        for name, prec in (("fp64", IGAMG_FP64), ("mixed", IGAMG_FP32_IR)):
            t0 = time.perf_counter()
            S = Solver(p, n, L, sigma, 1.0, precision=prec, dim=3)
            setup = time.perf_counter() - t0
            F = S.load_vector(f)
            U = S.empty()
            for _ in range(args.warmup):
                U.zero_()
                S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
            ts = []
            for _ in range(args.steps):
                U.zero_()
                dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False), stream)
                assert rep["converged"], rep
                ts.append(dt)
            t = sum(ts) / len(ts)
            sz = S.sizes()
            sweeps = 4
            dt_sm, _ = _timed(lambda: S.smooth(U, F, sweeps=sweeps), stream)
            out["%s_sigma%g" % (name, sigma)] = {
                "solve_ms": 1e3 * t, "cycles": rep["cycles"], "rel_residual": rep["rel_residual"],
                "mdof_per_s_per_cycle": S.ndof() * rep["cycles"] / t / 1e6, "div_inf": rep["div_inf"],
                "setup_s": setup, "fine_sweep_ms": 1e3 * dt_sm / sweeps, "colours": sz.n_colours}
            S.close()
    line = {"metric": "3D solve time to 1e-8 rel. residual & MDOF/s per V-cycle (64^3 cube)", "workload": "cube",
            "config": {"workload": "3D generalized Stokes, unit cube, p=2 (velocity S^{2,1,1} x S^{1,2,1} x S^{1,1,2}), "
                                   "64^3 elements, 5 levels, sigma/nu in {1, 1e3}, manufactured forcing of Sec. 6.3, "
                                   "V(2,2) multiplicative vector-potential Schwarz, zero initial guess, to 1e-8",
                       "ndof": 3 * 64 * 65 * 65 + 65 ** 3 + 1}, "results": out}
    print(json.dumps(line), flush=True)


def run_cube_oseen(args):
    """3D generalized Oseen on the unit cube (the regimes of Table 7): p = 2, 64^3 elements,
    5 grids, beta = the manufactured velocity scaled to max |beta| = 1, (Re, Da) = (1, 1) with
    nu = 1, sigma = 1 and (100, 1000) with nu = 0.01, sigma = 10; manufactured forcing;
    FP64 and FP32-in-FP64 solves from zero to 1e-8 (per-row operator records in HBM)."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR, IGAMG_FP64
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 64, 5
    beta = inputs.oseen_advection_3d(p, n, 1.0)
    stream = torch.cuda.current_stream()
    out = {}
    for re_, da, sigma, nu in ((1, 1, 1.0, 1.0), (100, 1000, 10.0, 0.01)):
        f = torch.tensor(inputs.oseen_forcing_3d(p, n, sigma, nu, beta), device="cuda")
        for name, prec in (("fp64", IGAMG_FP64), ("mixed", IGAMG_FP32_IR)):
            t0 = time.perf_counter()
            S = Solver(p, n, L, sigma, nu, precision=prec, dim=3, beta=beta)
            setup = time.perf_counter() - t0
            F = S.load_vector(f)
            U = S.empty()
            for _ in range(args.warmup):
                U.zero_()
                S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
            ts = []
            for _ in range(args.steps):
                U.zero_()
                dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False), stream)
                assert rep["converged"], rep
                ts.append(dt)
            t = sum(ts) / len(ts)
            out["%s_Re%d_Da%d" % (name, re_, da)] = {
                "solve_ms": 1e3 * t, "cycles": rep["cycles"], "rel_residual": rep["rel_residual"],
                "mdof_per_s_per_cycle": S.ndof() * rep["cycles"] / t / 1e6, "div_inf": rep["div_inf"],
                "setup_s": setup}
            S.close()
    line = {"metric": "3D Oseen solve time to 1e-8 rel. residual (Table 7 regimes)", "workload": "cube-oseen",
            "config": {"workload": "3D generalized Oseen, unit cube, p=2, 64^3 elements, 5 levels, max|beta|=1, "
                                   "(Re, Da) in {(1, 1), (100, 1000)}, manufactured forcing, V(2,2) multiplicative",
                       "ndof": 3 * 64 * 65 * 65 + 65 ** 3 + 1}, "results": out}
    print(json.dumps(line), flush=True)


def run_smoothers(args):
    """Additive (eq. ASM) against multiplicative (eq. MSM) Schwarz at the headline size:
    2D generalized Stokes, 256 x 256, 7 grids, p = 2 and 3, sigma = nu = 1, GRF forcing,
    FP64, V(2,2), zero guess, to 1e-8 (the trade-off of the paper's Tables 1 and 2: the
    additive sweep is three launches, the multiplicative one (p+1)^2)."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IgamgError
    from paper_1705_09282_gb300.solver import Solver
    stream = torch.cuda.current_stream()
    out = {}
    for p in DEGREES:
        f = torch.tensor(inputs.grf_forcing(p, N_FINE, seed=SEED), device="cuda")
        for name, sm, eta in (("mult", "mult", 0.5), ("add_eta0.3", "add", 0.3), ("add_eta0.2", "add", 0.2)):
            S = Solver(p, N_FINE, N_LEVELS, 1.0, 1.0, smoother=sm, eta=eta, nu1=2, nu2=2)
            F = S.load_vector(f)
            U = S.empty()
            ts = []
            try:
                for _ in range(args.warmup):
                    U.zero_()
                    S.solve(U, F, rtol=RTOL, max_cycles=200, history=False)
                for _ in range(args.steps):
                    U.zero_()
                    dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=200, history=False), stream)
                    ts.append(dt)
            except IgamgError as e:          # eq. ASM can diverge (reading R9): report it
                out["p%d_%s" % (p, name)] = {"converged": False, "error": str(e)}
                S.close()
                continue
            t = sum(ts) / len(ts)
            out["p%d_%s" % (p, name)] = {"converged": rep["converged"], "cycles": rep["cycles"], "solve_ms": 1e3 * t,
                                         "ms_per_cycle": 1e3 * t / max(rep["cycles"], 1), "div_inf": rep["div_inf"]}
            S.close()
    line = {"metric": "additive vs multiplicative Schwarz: solve time to 1e-8", "workload": "smoothers",
            "config": {"workload": "2D generalized Stokes, 256x256, 7 levels, p=2,3, sigma=nu=1, GRF forcing, FP64, V(2,2)"},
            "results": out}
    print(json.dumps(line), flush=True)


def run_annulus(args):
    """Generalized Stokes on the quarter annulus (Sec. 6.2's domain, r = 0.075 .. 0.225,
    push-forward spaces of Sec. 4.3): p = 2, 256 x 256 elements, 7 grids, sigma/nu in
    {1, 1e3}, the closed-form manufactured forcing, V(2,2) multiplicative, zero guess, to
    1e-8; FP64, FP32-in-FP64 and FGMRES.  The operator is stored per row (three boxes,
    u_x - u_y coupled) and every patch has its own inverse, so the sweeps stream their
    records from HBM."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import (IGAMG_FGMRES_FP64, IGAMG_FP32_IR, IGAMG_FP64,
                                             IGAMG_GEOM_QUARTER_ANNULUS, IgamgError)
    from paper_1705_09282_gb300.solver import Solver
    p, n, L, nu = 2, N_FINE, N_LEVELS, 1.0
    stream = torch.cuda.current_stream()
    out = {}
    for sigma in (1.0, 1e3):
        for name, prec in (("fp64", IGAMG_FP64), ("fp32-in-fp64", IGAMG_FP32_IR), ("fgmres", IGAMG_FGMRES_FP64)):
            key = "sigma%g_%s" % (sigma, name)
            t0 = time.perf_counter()
            try:
                S = Solver(p, n, L, sigma, nu, precision=prec, geometry=IGAMG_GEOM_QUARTER_ANNULUS)
            except IgamgError as e:
                out[key] = {"error": str(e)}
                continue
            setup = time.perf_counter() - t0
            X = S.quad_points_xy()
            F = S.load_vector(torch.tensor(inputs.annulus_forcing(X[0], X[1], sigma, nu), device="cuda"))
            U = S.empty()
            for _ in range(args.warmup):
                U.zero_()
                S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False)
            ts = []
            for _ in range(args.steps):
                U.zero_()
                dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=MAXC, history=False), stream)
                ts.append(dt)
            t = sum(ts) / len(ts)
            r = {"converged": rep["converged"], "cycles": rep["cycles"], "solve_ms": 1e3 * t,
                 "mdof_per_s_per_cycle": S.ndof() * rep["cycles"] / t / 1e6, "div_inf": rep["div_inf"],
                 "setup_s": setup}
            if name == "fp64":
                sz = S.sizes()
                sweeps = 10
                dt_sm, _ = _timed(lambda: S.smooth(U, F, sweeps=sweeps), stream)
                r["fp64_colour_launch_us"] = 1e6 * dt_sm / (sweeps * sz.n_colours)
                R = S.empty()
                dt_r, _ = _timed(lambda: [S.residual(U, F, out=R) for _ in range(20)], stream)
                res_us = 1e6 * dt_r / 20
                RU = (2 * p + 1) * (2 * p - 1) + 2 * p * (2 * p - 1) + 1
                nvel = sz.n_ux + sz.n_uy
                res_bytes = (sz.n_total - 1) * (RU * 8 + 3 * 8) + nvel * 4 * p * p * 8
                pk, src = peaks()
                r["fp64_residual_us"] = res_us
                r["residual_hbm"] = {"bytes": res_bytes, "achieved_gbs": res_bytes / res_us / 1e3,
                                     "peak_gbs": pk["hbm_gbs"], "frac": res_bytes / res_us / 1e3 / pk["hbm_gbs"],
                                     "peak_source": src}
            out[key] = r
            S.close()
    line = {"metric": "solve time to 1e-8 rel. residual on the quarter annulus", "workload": "annulus",
            "config": {"workload": "2D generalized Stokes on the quarter annulus (r 0.075..0.225), p=2, 256x256, "
                                   "7 levels, sigma/nu in {1, 1e3}, manufactured forcing, V(2,2) multiplicative, "
                                   "zero guess, to 1e-8, set-up not timed"},
            "results": out}
    print(json.dumps(line), flush=True)


def run_cylinder(args):
    """Generalized Stokes on the hollow cylinder section (the quarter annulus extruded by 0.1,
    push-forward spaces of Sec. 4.3): p = 2, n^3 elements for each n in --cyl-n (default 16),
    coarsest grid 4^3, sigma = nu = 1, the closed-form manufactured forcing, V(2,2)
    multiplicative, zero guess, to 1e-8 (at most 400 cycles: the V-cycle count grows with n
    here); FP64, FP32-in-FP64 and FGMRES.  Set-up (host assembly
    on the mapped cube) is not timed."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import (IGAMG_FGMRES_FP64, IGAMG_FP32_IR, IGAMG_FP64,
                                             IGAMG_GEOM_HOLLOW_CYLINDER)
    from paper_1705_09282_gb300.solver import Solver
    stream = torch.cuda.current_stream()
    out = {}
    sizes = [int(v) for v in str(args.cyl_n).split(",")]
    for n, (name, prec) in ((n, c) for n in sizes for c in (("fp64", IGAMG_FP64), ("fp32-in-fp64", IGAMG_FP32_IR),
                                                             ("fgmres", IGAMG_FGMRES_FP64))):
        levels = max(1, (n // 4).bit_length())
        t0 = time.perf_counter()
        S = Solver(2, n, levels, 1.0, 1.0, dim=3, precision=prec, geometry=IGAMG_GEOM_HOLLOW_CYLINDER)
        setup = time.perf_counter() - t0
        X = S.quad_points_xy()
        F = S.load_vector(torch.tensor(inputs.cylinder_forcing(X[0], X[1], X[2], 1.0, 1.0), device="cuda"))
        U = S.empty()
        for _ in range(args.warmup):
            U.zero_()
            S.solve(U, F, rtol=RTOL, max_cycles=400, history=False)
        ts = []
        for _ in range(args.steps):
            U.zero_()
            dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=400, history=False), stream)
            ts.append(dt)
        t = sum(ts) / len(ts)
        key = name if len(sizes) == 1 else f"{n}^3 {name}"
        out[key] = {"converged": rep["converged"], "cycles": rep["cycles"], "solve_ms": 1e3 * t,
                    "div_inf": rep["div_inf"], "setup_s": setup, "ndof": S.ndof(), "levels": levels}
        S.close()
    line = {"metric": "solve time to 1e-8 rel. residual on the hollow cylinder section", "workload": "cylinder",
            "config": {"workload": "3D generalized Stokes on the hollow cylinder section (quarter annulus r 0.075..0.225 "
                                   f"extruded by 0.1), p=2, n^3 for n in {sizes}, coarsest 4^3, sigma=nu=1, "
                                   "manufactured forcing, V(2,2) multiplicative, zero guess, to 1e-8, set-up not timed"},
            "results": out}
    print(json.dumps(line), flush=True)


def run_cycles(args):
    """Cycle forms on the harder cases (the W-cycle and full multigrid that Sec. 5's opening
    paragraph names, and FGMRES around the V-cycle): 3D generalized Stokes on the 64^3 cube;
    2D generalized Stokes at 256 x 256,
    7 grids, p = 2, 3, sigma/nu = 1e-4 and 1e4; generalized Oseen at 512 x 512, 8 grids,
    nu = 1e-2, sigma = 1, max|beta| = 0.5 and 1 (Re = 50 and 100); GRF forcing, V(2,2)
    multiplicative, FP64, zero guess, to 1e-8.  Set-up is not timed."""
    import torch

    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300._lib import IGAMG_FGMRES_FP64, IGAMG_FP32_IR, IGAMG_FP64, IgamgError
    from paper_1705_09282_gb300.solver import Solver
    stream = torch.cuda.current_stream()
    forms = (("V", dict(gamma=1, fmg=False, precision=IGAMG_FP64)),
             ("W", dict(gamma=2, fmg=False, precision=IGAMG_FP64)),
             ("FMG+V", dict(gamma=1, fmg=True, precision=IGAMG_FP64)),
             ("FMG+W", dict(gamma=2, fmg=True, precision=IGAMG_FP64)),
             ("FGMRES(V)", dict(gamma=1, fmg=False, precision=IGAMG_FGMRES_FP64)),
             ("FMG+V fp32-in-fp64", dict(gamma=1, fmg=True, precision=IGAMG_FP32_IR)))
    cases = [("cube p2 sigma1", 2, 64, 5, 1.0, 1.0, "cube", None),
             ("stokes p2 sigma1e-4", 2, N_FINE, N_LEVELS, 1e-4, 1.0, None, SEED),
             ("stokes p3 sigma1e-4", 3, N_FINE, N_LEVELS, 1e-4, 1.0, None, SEED),
             ("stokes p3 sigma1e4", 3, N_FINE, N_LEVELS, 1e4, 1.0, None, SEED),
             ("oseen Re50", 2, 512, 8, 1.0, 1e-2, 0.5, 1707),
             ("oseen Re100", 2, 512, 8, 1.0, 1e-2, 1.0, 1707)]
    out = {}
    for name, p, n, L, sigma, nu, bmax, seed in cases:
        cube = bmax == "cube"
        beta = inputs.oseen_advection(p, n, bmax) if (bmax and not cube) else None
        f = torch.tensor(inputs.manufactured_forcing_3d(p, n, sigma, nu) if cube else inputs.grf_forcing(p, n, seed=seed),
                         device="cuda")
        res = {}
        for fname, kw in forms:
            try:
                S = Solver(p, n, L, sigma, nu, beta=beta, dim=3 if cube else 2, **kw)
            except IgamgError as e:
                res[fname] = {"error": str(e)}
                continue
            F = S.load_vector(f)
            U = S.empty()
            try:
                for _ in range(args.warmup):
                    U.zero_()
                    S.solve(U, F, rtol=RTOL, max_cycles=100, history=False)
                ts = []
                for _ in range(args.steps):
                    U.zero_()
                    dt, rep = _timed(lambda: S.solve(U, F, rtol=RTOL, max_cycles=100, history=False), stream)
                    ts.append(dt)
                t = sum(ts) / len(ts)
                res[fname] = {"converged": rep["converged"], "cycles": rep["cycles"], "solve_ms": 1e3 * t,
                              "rel_residual": rep["rel_residual"], "div_inf": rep["div_inf"]}
            except IgamgError as e:          # a divergent form reports a non-finite residual
                res[fname] = {"converged": False, "error": str(e)}
            S.close()
        out[name] = res
    line = {"metric": "solve time and cycles to 1e-8 for the V-, W- and full-multigrid cycles and FGMRES",
            "workload": "cycles",
            "config": {"workload": "3D generalized Stokes 64^3 (5 levels, p=2, sigma=nu=1, manufactured forcing), "
                                   "2D generalized Stokes 256x256 (7 levels, p=2,3, sigma/nu=1e-4,1e4) and Oseen "
                                   "512x512 (8 levels, nu=1e-2, sigma=1, max|beta|=0.5,1), GRF forcing, V(2,2) "
                                   "multiplicative, zero guess, to 1e-8, set-up not timed"},
            "results": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="stokes",
                    choices=["stokes", "oseen", "batch", "cube", "cube-oseen", "smoothers", "cycles", "annulus",
                             "cylinder"],
                    help="stokes: the headline sweep (default); the others: extra measurements")
    ap.add_argument("--batch-count", type=int, default=1024)
    ap.add_argument("--cyl-n", default="16", help="cylinder workload: comma-separated mesh sizes (n^3)")
    ap.add_argument("--train-count", type=int, default=384)
    ap.add_argument("--train-steps", type=int, default=6000)
    ap.add_argument("--profile-case", default=None,
                    help="run two untimed solves of one case (for ncu), e.g. p2-fp64 or p2-mixed")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "oseen":
        run_oseen(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "cube":
        run_cube(args)
    elif args.workload == "smoothers":
        run_smoothers(args)
    elif args.workload == "cube-oseen":
        run_cube_oseen(args)
    elif args.workload == "cycles":
        run_cycles(args)
    elif args.workload == "annulus":
        run_annulus(args)
    elif args.workload == "cylinder":
        run_cylinder(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
