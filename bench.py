"""Benchmark: particle-steps/s of the IFE-PIC hot path, including the IFE solve.

Workload (default): the 64^3-cell sphere-charging problem -- 64^3 cubic cells of
0.5 Debye length (1.31M tets), sphere radius 6 centred, eps 4 inside, e- and H+
(mass ratio 100) at 64 particles/cell/species (~33.5M particles), phi = 0 on
the faces, Maxwellian flux injection, dt = 0.05.  One step = push + object
collection + injection + rebin + scatter + IFE PCG solve + node field.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica (the method's single-GPU path does not shard) and rank 0 prints the
aggregate; the reference arm runs on rank 0 only.
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

PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# the headline metric: `value` is the plain (single-instance) rate; the line's `batched` and `served`
# objects carry the batched rate (and its ratio to the plain one) and the served p50/p99 latency
METRIC = "particle-steps/s incl. IFE solve, batched vs plain; served p50/p99 latency"
PROFILE_RANGE = False   # --profile-range: profiler start/stop around the timed steps (ncu --profile-from-start off)
BIN_EDGE = None   # MIXED particle-bin edge of the measured contexts (--bin-edge; None = the library's default)
PRECOND = 0   # MIXED preconditioner of the measured contexts (--precond; 0 = the library's automatic choice)
BYTES_PER_PARTICLE_STEP = {"fp64": 96, "mixed": 56}     # read + write of the particle state
E2E_PASSES = 3   # end-to-end passes; the median is reported


def _peaks():
    try:
        with open(PEAKS) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """SM clock and clock-event reasons sampled during the timed region: NVML
    through ctypes every 2 ms (the driver's library; reads only), else
    nvidia-smi every 200 ms."""

    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, index=0):
        self.p = None
        self.nvml = None
        self.sm, self.mx, self.reasons = [], [], set()
        try:
            self._start_nvml(index)
        except Exception:
            self.nvml = None
            self._start_smi(index)

    def _start_nvml(self, index):
        import ctypes
        import threading
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        dev = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(dev)) != 0:
            raise RuntimeError("nvml handle")
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0:
            self.mx.append(float(mx.value))
        self.nvml = lib
        self.stop_flag = False

        def run():
            clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
            while not self.stop_flag:
                if lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0:
                    self.sm.append(float(clk.value))
                if get_reasons(dev, ctypes.byref(rs)) == 0:
                    for bit, nm in self.REASONS.items():
                        if rs.value & bit:
                            self.reasons.add(nm)
                time.sleep(0.002)

        self.th = threading.Thread(target=run, daemon=True)
        self.th.start()

    def _start_smi(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.nvml is not None:
            self.stop_flag = True
            self.th.join(timeout=5)
            try:
                self.nvml.nvmlShutdown()
            except Exception:
                pass
            sm = self.sm
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(self.mx) if self.mx else None,
                    "reasons": sorted(self.reasons), "samples": len(sm), "sampler": "nvml 2 ms"}
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "sampler": "nvidia-smi 200 ms"}


def workload(name):
    from paper_2011_10214_gb300 import workloads as wl
    return {"sphere64": wl.SPHERE64, "sphere16": wl.SPHERE16,
            "sphere32": wl.sphere_config(32, 3.0, 64, 100, seed_offset=6),
            "crater160": wl.CRATER160,
            "crater80": wl.crater_config(80, 80, 40, 10.0, 15.0, 5.0, seed_offset=7),
            "oml50": wl.OML50,
            "sphere64h2": dict(wl.SPHERE64, name="sphere64h2", ife_refine=2),
            "lunar200": wl.LUNAR200,
            "lunar100": wl.lunar_config(100, 50, 50, 4.75, 2.25, 5.25, 10.1, 15.45, 1.35, 2.0, seed_offset=9)}[name]


def cfg_desc(cfg, precision, extra=None):
    n = cfg["n"]
    ppc = cfg["species"][0]["ppc"]
    ob = cfg["object"]
    if ob["kind"] == "rim_crater":
        w = (f"lunar crater charging {n[0]}x{n[1]}x{n[2]} cells (h={cfg['h']}), half raised-rim crater (radii "
             f"{ob['r_inner']}/{ob['r_top']}/{ob['r_outer']}, rim {ob['height']} above and floor {ob['depth']} below "
             f"the ground) in regolith eps {ob['eps_in']} at z={ob['z_ground']} over bedrock eps "
             f"{ob['bedrock'][1]} below z={ob['bedrock'][0]}, {ppc} ppc/species solar-wind e-+H+ drifting 8 v_ti "
             f"at 10 deg, photoelectrons (sun 10 deg above the ground), reflecting Y_min, injection at X_min/X_max/"
             f"Y_max/Z_max, dt={cfg['dt']}, phi=0 at Z_max, Neumann elsewhere")
    elif ob["kind"] == "cap_crater":
        w = (f"crater charging {n[0]}x{n[1]}x{n[2]} cells (h={cfg['h']}), ground z={ob['z_ground']} eps "
             f"{ob['eps_in']}, spherical-cap crater rim radius {ob['rim_radius']} depth {ob['depth']}, "
             f"{ppc} ppc/species solar-wind e-+H+ drifting 8 v_ti at 45 deg, photoelectrons from the sunlit "
             f"unshadowed surface, dt={cfg['dt']}, phi=0 at Z_max, Neumann elsewhere")
    elif cfg.get("particle_bc"):
        w = (f"eighth-sphere OML sheath {n[0]}x{n[1]}x{n[2]} cells (h={cfg['h']}), R={ob['radius']} centred at "
             f"the origin corner, eps_in={ob['eps_in']}, {ppc} ppc/species e-+H+ "
             f"(m_i/m_e={cfg['species'][1]['m']:g}), dt={cfg['dt']}, zero-Neumann field and reflecting particle "
             f"faces at X/Y/Z_min, phi=0 and flux injection at X/Y/Z_max")
    else:
        w = (f"sphere charging {n[0]}x{n[1]}x{n[2]} cells (h={cfg['h']}), R={ob['radius']}, "
             f"eps_in={ob['eps_in']}, {ppc} ppc/species e-+H+ (m_i/m_e={cfg['species'][1]['m']:g}), "
             f"dt={cfg['dt']}, flux injection, phi=0 faces")
    if cfg.get("ife_refine", 1) > 1:
        r = cfg["ife_refine"]
        w += (f"; hybrid grid: IFE mesh {r * n[0]}x{r * n[1]}x{r * n[2]} cells (h={cfg['h'] / r}), the PIC "
              f"mesh refined {r}x per axis")
    d = {"workload": w,
         "precision": precision, "pcg_tol": 1e-6, "pcg_max_iter": 150,
         "l2_flush": "inputs larger than L2 (particle state > 1 GB per step)"}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------
# FP64 push, from an ncu capture of one k_push_bins launch on the 32^3 sphere (4,076,523 particles):
# sm__inst_executed_pipe_fp64.sum = 18,357,080 warp instructions (4.50 per particle, 144 lane operations),
# DADD 183,285,395 + DMUL 256,496,282 + DFMA 9,065 thread instructions (107.9 flops per particle; the kernel
# keeps DADD and DMUL apart, no FMA contraction, for results bit-identical to the FP64 oracle)
FP64_PIPE_WARP_INST_PER_PARTICLE = 18357080 / 4076523
FP64_FLOPS_PER_PARTICLE_STEP = (183285395 + 256496282 + 2 * 9065) / 4076523
FP64_LANES_PER_CLK_SM = 2              # FP64 pipe: 2 lane operations per clock per SM (GB300)
# PCG: 7 node-vector passes per iteration (p, x, r, z updates, the operator's read of p and write of q)
SOLVE_BYTES_PER_NODE_ITER = {"mixed": 7 * 4, "fp64": 7 * 8}
# DRAM bytes per pushed particle of one k_push_bins_m launch, from an ncu capture of the 64^3 sphere
# bench workload (dram__bytes_read.sum + dram__bytes_write.sum over the launch's particles); None when
# not measured for the current kernel
PUSH_TRAFFIC_PER_PARTICLE = {"mixed": (930762240 + 860456448) / 32619866, "fp64": None}
NSM, DFMA_PER_CLK_SM = 152, 2          # GB300: 2 FP64 FMA per SM per clock


def measure(cfg, precision, steps, warmup, stream, dist, local):
    """Set up one instance, warm up, time `steps` PIC steps with CUDA events."""
    import torch
    from paper_2011_10214_gb300 import capi
    prec = capi.MIXED if precision == "mixed" else capi.FP64
    sim = capi.from_config(cfg, precision=prec, stream=stream.cuda_stream,
                           bin_edge=BIN_EDGE if prec == capi.MIXED else None)
    if PRECOND:
        sim.set_preconditioner(PRECOND)
    sim.solve()
    sim.leapfrog_init()
    if warmup > 0:
        sim.step(warmup)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    barrier()
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if PROFILE_RANGE:
        torch.cuda.profiler.start()
    ev0.record(stream)
    st = sim.step(steps)
    ev1.record(stream)
    barrier()
    if PROFILE_RANGE:
        torch.cuda.profiler.stop()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    pushed = sum(st["pushed"])
    secs, total = combine_ranks(ms / 1e3, pushed, dist, "cuda")
    return sim, st, secs, total, pushed, ck


def combine_ranks(seconds, pushed, dist, device):
    """Whole-job figures of the replicas: the slowest rank's time (max over
    ranks) and the particle-steps of all ranks (sum); one rank's own without
    a process group."""
    import torch
    if dist is None:
        return float(seconds), float(pushed)
    tmax = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    tsum = torch.tensor([float(pushed)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def roofline(precision, st, steps, ck):
    """Dominant kernel: the fused gather/push/collect/deposit launch (phase 0)."""
    push_ms = st["phase_ms"][0] / steps
    per_launch = sum(st["pushed"]) / steps
    peaks, src = _peaks()
    if precision == "mixed":
        alg = per_launch * BYTES_PER_PARTICLE_STEP["mixed"]
        ach = alg / (push_ms / 1e3) / 1e9
        tpp = PUSH_TRAFFIC_PER_PARTICLE["mixed"]
        return {"kernel": "k_push_bins_m (fused gather+push+collect+deposit, FP32 state)", "bound": "hbm",
                "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 4),
                "traffic": None if tpp is None else round(tpp * per_launch),
                "traffic_note": "ncu DRAM bytes per particle of a 64^3 sphere launch (54.9 B, 0.98 of the "
                                "algorithmic 56 B), scaled to this launch's particles",
                "peak_source": src, "alg_bytes_per_launch": alg, "avg_launch_ms": push_ms}
    # bound by the FP64 pipe: its lane operations (every FP64-pipe warp instruction x 32 lanes: DADD, DMUL,
    # conversions, compares, roundings) per second against 152 SMs x 2 lanes/clk x max SM clock
    mhz = peaks.get("sm_max_mhz", 2070.0)
    ops = per_launch * FP64_PIPE_WARP_INST_PER_PARTICLE * 32
    ach = ops / (push_ms / 1e3) / 1e9
    peak = NSM * FP64_LANES_PER_CLK_SM * mhz / 1e3
    flops = per_launch * FP64_FLOPS_PER_PARTICLE_STEP
    return {"kernel": "k_push_bins (FP64, no FMA contraction)", "bound": "alu", "achieved": round(ach, 1),
            "peak": round(peak, 1), "unit": "G FP64-pipe ops/s", "frac": round(ach / peak, 4), "traffic": None,
            "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x max SM clock",
            "ops_per_particle_step": round(FP64_PIPE_WARP_INST_PER_PARTICLE * 32, 1),
            "flops_view": {"achieved_gflops": round(flops / (push_ms / 1e3) / 1e9, 1),
                           "flops_per_particle_step": round(FP64_FLOPS_PER_PARTICLE_STEP, 1),
                           "peak_gflops_with_fma": round(NSM * DFMA_PER_CLK_SM * 2 * mhz / 1e3, 1)},
            "avg_launch_ms": push_ms,
            "hbm_view": {"achieved_gbs": round(per_launch * 96 / (push_ms / 1e3) / 1e9, 1),
                         "peak_gbs": peaks["hbm_gbs"]}}


def roofline_solve(precision, st, steps, nnodes, solver):
    """The field solve: algorithmic node-vector bytes of the PCG iterations over the solve graph's time
    (the persistent PCG kernel plus the short RHS, start-vector and node-field kernels around it)."""
    solve_ms = st["phase_ms"][5] / steps
    iters = st["pcg_iters_total"] / steps
    alg = nnodes * SOLVE_BYTES_PER_NODE_ITER[precision] * iters
    ach = alg / (solve_ms / 1e3) / 1e9
    peaks, src = _peaks()
    # the solver the library ran (pifepic_get_solver: 1 registers, 2 global memory, 3 multigrid)
    reg, mg = solver == 1, solver == 3
    if mg:
        # per inner iteration: the PCG's 7 FP32 passes plus the V-cycle's fine-level passes (pre-smoothing
        # 12 B, residual 12 B, correction 8 B, post-smoothing 16 B); the coarse levels add about 1/7 more
        alg = nnodes * (SOLVE_BYTES_PER_NODE_ITER["mixed"] + 48) * iters
        ach = alg / (solve_ms / 1e3) / 1e9
    kname = ("k_pcg_mg (global memory, multigrid V-cycle)" if mg else
             "k_pcg_reg (registers)" if reg else "k_pcg_glob (global memory)")
    return {"kernel": f"{kname}: persistent PCG, one launch per solve, in the solve graph", "bound": "hbm",
            "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": None, "peak_source": src,
            "alg_bytes_per_launch": alg, "avg_launch_ms": solve_ms, "iters_per_solve": iters,
            "note": ("multigrid-preconditioned PCG: ~16-20 grid barriers per inner iteration, vectors in L2" if mg else
                     "latency-bound: one grid exchange per inner iteration (pipelined PCG), vectors in registers "
                     "and L2" if precision == "mixed" else
                     "latency-bound: two grid exchanges per iteration, vectors in registers and L2")}


def run_gpu(args):
    import numpy as np
    import torch
    from paper_2011_10214_gb300 import capi

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = workload(args.workload)
    stream = torch.cuda.Stream()
    main = args.precision
    other = "fp64" if main == "mixed" else "mixed"
    sim, st, secs, total, pushed, ck = measure(cfg, main, args.steps, args.warmup, stream, dist, local)
    value = total / secs
    nnodes = sim.sizes()["nnodes"]
    roof_push = roofline(main, st, args.steps, ck)
    roof_solve = roofline_solve(main, st, args.steps, nnodes, sim.solver)
    # the longer of the two phases is the dominant kernel; the other is reported beside it
    if roof_solve["avg_launch_ms"] > roof_push["avg_launch_ms"]:
        roof, roof_other = roof_solve, roof_push
    else:
        roof, roof_other = roof_push, roof_solve

    # end to end through the C ABI from host buffers: the initial particle state
    # is copied host -> device (pinned) inside the timed region, and every step
    # reads the potential and the step statistics back to host memory
    e2e = None
    if not args.no_e2e:
        state = [sim.particles(s) for s in range(len(cfg["species"]))]
        prec = capi.MIXED if main == "mixed" else capi.FP64
        pinned = []
        for P in state:
            pinned.append({k: torch.from_numpy(np.ascontiguousarray(P[k])).pin_memory().numpy()
                           for k in ("x", "y", "z", "vx", "vy", "vz")})
        h2d = sum(P[k].nbytes for P in pinned for k in P)
        # three passes, each on a fresh context (a host-timed region is exposed to
        # the host's own hiccups); the median is reported
        rates = []
        for _pass in range(E2E_PASSES):
            sim2 = capi.from_config(cfg, precision=prec, stream=stream.cuda_stream, load=False)
            nn = sim2.sizes()["nnodes"]
            phi_host = torch.empty(nn, dtype=torch.float64).pin_memory().numpy()
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            for s, P in enumerate(pinned):
                sim2.load_particles(s, P["x"], P["y"], P["z"], P["vx"], P["vy"], P["vz"])
            sim2.solve()
            pushed2 = 0
            for _ in range(args.steps):
                st2 = sim2.step(1)
                pushed2 += sum(st2["pushed"])
                capi.lib.pifepic_get_potential(sim2._c, phi_host.ctypes.data, capi.HOST)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            secs2, total2 = combine_ranks(t1 - t0, pushed2, dist, "cuda")   # the whole job over the replicas
            rates.append(total2 / secs2)
            sim2.close()
        e2e = {"value": sorted(rates)[len(rates) // 2], "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(world * h2d / args.steps),
               "d2h_bytes_per_step": int(world * (phi_host.nbytes + 512)),
               "passes": [round(r, 1) for r in rates],
               "note": "median of %d passes, each on a fresh context: initial particle state h2d (amortised over "
                       "the steps), the initial solve, then per step the step and the phi and stats d2h; the "
                       "replicas' particle-steps over the slowest rank's time" % E2E_PASSES}
    sim.close()

    # the other precision on the same workload, for the FP32-refined vs plain FP64 comparison
    alt = None
    if not args.no_compare:
        sim_b, st_b, secs_b, total_b, _, ck_b = measure(cfg, other, args.steps, args.warmup, stream, dist, local)
        alt = {"precision": other, "value": total_b / secs_b, "ms_per_step": secs_b * 1e3 / args.steps,
               "roofline": roofline(other, st_b, args.steps, ck_b),
               "pcg_iters_per_step": st_b["pcg_iters_total"] / args.steps,
               "phase_ms_per_step": {k: v / args.steps for k, v in zip(PHASES, st_b["phase_ms"]) if v}}
        sim_b.close()

    out = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main == "fp64" else "f32+f64",
        "data": "synthetic (seeded Philox load and injection)",
        "config": cfg_desc(cfg, main, {"particles": int(pushed / args.steps),
                                       "parallelism": f"replicas x{world}",
                                       "bin_edge": BIN_EDGE or 4}),
        "roofline": roof, "roofline_other": roof_other, "clocks": ck, "e2e": e2e,
        "gpu_launches": int(st["kernel_launches"]),
        "pcg_iters_per_step": st["pcg_iters_total"] / args.steps,
        "pcg_refinements_per_step": st["pcg_outer_total"] / args.steps,
        "events_per_step": {k: [round(v / args.steps, 1) for v in st[k]]
                            for k in ("pushed", "absorbed", "collected", "injected") if k in st},
        "phase_ms_per_step": {k: v / args.steps for k, v in zip(PHASES, st["phase_ms"]) if v},
        "compare": alt,
    }
    # the metric's batched and served parts (rank 0, one GPU each; bounded)
    if rank == 0 and not args.no_batched and args.workload == "sphere64":
        b = measure_batch(args.instances, args.steps, args.warmup)
        b["vs_plain"] = b["value"] / value
        out["batched"] = b
    if rank == 0 and not args.no_served and args.workload == "sphere64":
        out["served"] = measure_serve(args.rate, args.served_horizon, args.max_steps, args.time_limit,
                                      args.hbm_budget_gb, True)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_subprocess(args)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


PHASES = ("push", "movers", "inject", "rebin", "rhs", "solve", "node_E", "other")


# ---------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------
def oracle_rate(workload_name, sample_frac, steps):
    """Time the oracle on a bounded sample: the full mesh and IFE solve, a
    random 1/sample_frac of the particles.  Particle work scales with the
    particle count, so the rate at full size is extrapolated as
    N / (t_particles * N / n_sample + t_field)."""
    from oracle.geometry import CapCrater, Mesh, NoObject, RimCrater, Sphere, set_bedrock
    from oracle.pic import Simulation
    from paper_2011_10214_gb300 import workloads as wl
    cfg = workload(workload_name)
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    if ob["kind"] == "sphere":
        obj = Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"])
    elif ob["kind"] == "cap_crater":
        obj = CapCrater(m, ob["z_ground"], ob["xc"], ob["yc"], ob["rim_radius"], ob["depth"], ob["eps_in"],
                        ob["eps_out"])
    elif ob["kind"] == "rim_crater":
        obj = RimCrater(m, ob["z_ground"], ob["xc"], ob["yc"], ob["r_inner"], ob["r_top"], ob["r_outer"],
                        ob["height"], ob["depth"], ob["eps_in"], ob["eps_out"])
    else:
        obj = NoObject()
    if ob.get("bedrock") is not None:
        set_bedrock(obj, m, *ob["bedrock"])
    sim = Simulation(m, obj, cfg["face_bc"], cfg["dt"], refine=cfg.get("ife_refine", 1))
    nfull = 0
    for s, sp in enumerate(cfg["species"]):
        sim.add_species(sp["q"], sp["m"], wl.macro_weight(cfg, sp))
        if cfg.get("particle_bc"):
            sim.set_particle_bc(s, cfg["particle_bc"])
        sim.load_maxwellian(s, sp["ppc"] // sample_frac if sp["ppc"] >= sample_frac else 1, sp["vth"], sp["drift"],
                            cfg["seed"])
        nfull += sp["ppc"] * m.ncells
        sim.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
        # injection at the sample's weight keeps the density; rates scale with 1/w
    ph = cfg.get("photo")
    if ph is not None:
        s = len(cfg["species"])
        sim.add_species(ph["q"], ph["m"], ph["weight"])
        if cfg.get("particle_bc"):
            sim.set_particle_bc(s, cfg["particle_bc"])
        sim.set_photoemission(s, ph["sun"], ph["density"], ph["vth"], cfg["seed"])
    sim.solve()
    sim.leapfrog_init()
    tp = tf = 0.0
    npush = 0
    for _ in range(steps):
        t0 = time.perf_counter()
        st = sim.step()
        t1 = time.perf_counter()
        npush += sum(st["pushed"])
        tp += t1 - t0
    # separate the field solve: time it once more on its own
    t0 = time.perf_counter()
    F = sim.node_load()
    phi, it, rr = sim.fs.solve(F, sim.qT, phi0=sim.phi, tol=sim.tol, maxit=sim.maxit)
    sim.fs.node_E(phi, sim.qT)
    tf = time.perf_counter() - t0
    tpart = max(tp / steps - tf, 1e-9)
    nsample = npush / steps
    full_step = tpart * nfull / nsample + tf
    return {"value": nfull / full_step, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{workload_name}: full mesh + IFE solve, {nsample:.0f} particles (1/{sample_frac} of the "
                      f"{nfull} load), {steps} steps; particle time scaled to the full count",
            "seconds": tp, "step_s": full_step}


def cpu_baseline_subprocess(args):
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "2", "--warmup", "0",
           "--workload", args.workload, "--as-baseline"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900,
                           env=dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1"))
        line = [l for l in r.stdout.splitlines() if l.startswith("{")][-1]
        d = json.loads(line)
        return d["cpu_baseline"]
    except Exception as e:
        return {"value": None, "error": str(e)[:200]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    frac = 16
    t0 = time.perf_counter()
    cb = oracle_rate(args.workload, frac, max(1, args.steps))
    t1 = time.perf_counter()
    cfg = workload(args.workload)
    out = {"impl": "reference", "metric": METRIC, "value": cb["value"],
           "unit": "particle-steps/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": cb["step_s"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Philox load and injection)", "config": cfg_desc(cfg, "fp64"),
           "cpu_baseline": dict(cb), "e2e": {"value": cb["value"], "unit": "particle-steps/s",
                                             "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": t1 - t0}
    print(json.dumps(out))


def measure_batch(instances, steps, warmup, autotune=True):
    """c4: `instances` independent sphere-charging instances (16^3..48^3 cells,
    R 1..8, eps 2..10, 16..64 ppc/species), MIXED, one graph launch per step;
    CUDA events on the batch stream around the timed steps."""
    import numpy as np
    import torch
    from paper_2011_10214_gb300 import capi, serve
    rng = np.random.default_rng(2011102144)
    cfgs = serve.request_distribution(rng, instances, big_fraction=0.0)
    stream = torch.cuda.Stream()
    # particle-bin edge per size class, by timing batches of each class (before the timed instances exist)
    tb = time.perf_counter()
    edges, edge_ms = serve.autotune_bin_edge(cfgs, stream=stream.cuda_stream) if autotune else ({}, {})
    tune_s = time.perf_counter() - tb
    t0 = time.perf_counter()
    sims = []
    for c in cfgs:
        s = capi.from_config(c, precision=capi.MIXED, stream=stream.cuda_stream,
                             bin_edge=edges.get(serve.size_class(c)))
        s.solve(); s.leapfrog_init()
        sims.append(s)
    setup_s = time.perf_counter() - t0
    # the same instances stepped one after another on their own (plain), for the batched-vs-plain ratio
    alone_ms, alone_pushed = 0.0, 0
    for s in sims:
        s.step(2, stats=False)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        sa = s.step(4)
        eb.record(stream)
        torch.cuda.synchronize()
        alone_ms += ea.elapsed_time(eb) / 4
        alone_pushed += sum(sa["pushed"]) / 4
    batch = capi.Batch(sims, stream=stream.cuda_stream)
    tuned = None
    if autotune:
        pc, cn, sps = serve.autotune_batch(batch)
        tuned = {"preconditioner": {capi.PRECOND_JACOBI: "jacobi", capi.PRECOND_MULTIGRID: "multigrid"}[pc],
                 "cta_nodes": cn, "trial_ms_per_step": sps * 1e3,
                 "bin_edge": {f"n{'<' if k[0] == 0 else '>='}32,ppc{('<=32', '<=48', '>48')[k[1]]}": e
                              for k, e in sorted(edges.items())},
                 "bin_edge_trial_ms": {f"{k[0]}{k[1]}": {str(e): round(t, 3) for e, t in v.items()}
                                       for k, v in sorted(edge_ms.items())},
                 "tune_s": tune_s}
    batch.step(warmup, stats=False)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if PROFILE_RANGE:
        torch.cuda.profiler.start()
    ev0.record(stream)
    st = batch.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if PROFILE_RANGE:
        torch.cuda.profiler.stop()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    pushed = sum(sum(x["pushed"]) for x in st)
    out = {"value": pushed / (ms / 1e3), "unit": "particle-steps/s", "ms_per_step": ms / steps, "steps": steps,
           "warmup": warmup, "instances": len(cfgs), "particles": int(pushed / steps),
           "workload": f"{len(cfgs)} independent sphere-charging instances, n ~ U{{16..48}}^3 cells (h=0.5), "
                       "R ~ U[1,8], eps ~ U[2,10], ppc ~ U{16..64} per species, MIXED, one graph launch per step",
           "tuner": tuned, "setup_s": setup_s,
           "alone": {"ms_per_step_sum": alone_ms, "value": alone_pushed / (alone_ms / 1e3),
                     "note": "the same instances stepped one after another, each alone (its own solve on "
                             "the whole GPU)"},
           "vs_alone": (alone_ms / (ms / steps)),
           "gpu_launches": int(sum(x["kernel_launches"] for x in st)), "graph_launches": steps,
           "pcg_iters_per_step_max": max(x["pcg_iters_total"] for x in st) / steps, "clocks": ck}
    batch.close()
    for s in sims:
        s.close()
    return out


def measure_serve(rate, horizon, max_steps, time_limit, hbm_budget_gb, overlap):
    """c5: Poisson arrivals of sphere-charging requests (the batched
    distribution plus 5 % at 96^3 with 64 ppc), admitted by HBM budget into one
    running batch; latency = finish - arrival (host clock)."""
    import numpy as np
    import torch
    from paper_2011_10214_gb300 import capi, serve
    rng = np.random.default_rng(2011102145)
    arr = serve.poisson_arrivals(rng, rate, horizon)
    reqs = serve.request_distribution(rng, len(arr), big_fraction=0.05)
    s_batch, s_admit = torch.cuda.Stream(), torch.cuda.Stream()
    srv = serve.Server(int(hbm_budget_gb * 2**30), precision=capi.MIXED, steps_per_round=10, max_steps=max_steps,
                       stream=s_batch.cuda_stream, overlap=overlap, admit_stream=s_admit.cuda_stream)
    res = srv.run(reqs, arr, time_limit=time_limit)
    srv.close()
    return {"p50_s": res["p50_s"], "p99_s": res["p99_s"], "completed": res["completed"], "requests": len(arr),
            "particle_steps_per_s": res["particle_steps_per_s"], "wall_s": res["wall_s"],
            "admission": "overlapped (worker thread, own stream)" if overlap else "synchronous (between rounds)",
            "workload": f"Poisson arrivals {rate}/s for {horizon} s; sphere-charging requests n ~ U{{16..48}}^3 "
                        f"(+5% 96^3 at 64 ppc), stop at {max_steps} steps or <1% change of the area-mean surface "
                        f"potential over 50 steps; HBM budget {hbm_budget_gb} GB"}


def run_batch(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    b = measure_batch(args.instances, args.steps, args.warmup, autotune=not args.no_autotune)
    out = {"metric": "particle-steps/s incl. IFE solve (batched)", "value": b["value"],
           "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": b["ms_per_step"], "higher_is_better": True, "dtype": "f32+f64",
           "data": "synthetic (seeded Philox load and injection)",
           "config": {"workload": b["workload"], "particles": b["particles"], "tuner": b["tuner"],
                      "setup_s": b["setup_s"]},
           "gpu_launches": b["gpu_launches"], "graph_launches": b["graph_launches"],
           "pcg_iters_per_step_max": b["pcg_iters_per_step_max"], "clocks": b["clocks"]}
    print(json.dumps(out))


def run_serve(args):
    """Both admission modes on the same arrival trace."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    modes = {"sync": [False], "overlap": [True], "both": [False, True]}[args.admission]
    res = [measure_serve(args.rate, args.horizon, args.max_steps, args.time_limit, args.hbm_budget_gb, o)
           for o in modes]
    main = res[-1]
    out = {"metric": "served latency p50/p99 and aggregate particle-steps/s", "unit": "s",
           "p50_s": main["p50_s"], "p99_s": main["p99_s"], "completed": main["completed"],
           "requests": main["requests"], "particle_steps_per_s": main["particle_steps_per_s"],
           "wall_s": main["wall_s"], "higher_is_better": False, "dtype": "f32+f64",
           "data": "synthetic (seeded Poisson arrivals)",
           "config": {"workload": main["workload"], "admission": main["admission"]},
           "runs": res}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="sphere64",
                    choices=["sphere64", "sphere32", "sphere16", "crater160", "crater80", "oml50", "lunar200",
                             "lunar100", "sphere64h2"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other precision's measurement")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve"])
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--no-autotune", action="store_true", help="batch: keep the default nodes per CTA of the clustered solves")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--horizon", type=float, default=60.0, help="serve mode: arrival horizon in seconds")
    ap.add_argument("--admission", default="both", choices=["sync", "overlap", "both"])
    ap.add_argument("--max-steps", type=int, default=500)
    ap.add_argument("--time-limit", type=float, default=600.0)
    ap.add_argument("--no-batched", action="store_true", help="default line: skip the batched (c4) part")
    ap.add_argument("--no-served", action="store_true", help="default line: skip the served (c5) part")
    ap.add_argument("--served-horizon", type=float, default=10.0, help="default line: served arrival horizon")
    ap.add_argument("--hbm-budget-gb", type=float, default=200.0)
    ap.add_argument("--as-baseline", action="store_true")
    ap.add_argument("--precond", default="auto", choices=["auto", "jacobi", "multigrid"],
                    help="MIXED field-solve preconditioner (pifepic_set_preconditioner)")
    ap.add_argument("--profile-range", action="store_true",
                    help="profiler start/stop around the timed steps (for ncu --profile-from-start off)")
    ap.add_argument("--bin-edge", type=int, default=None, choices=[4, 8],
                    help="MIXED particle bins of edge^3 cells (pifepic_set_bin_edge)")
    args = ap.parse_args()
    global PRECOND, BIN_EDGE, PROFILE_RANGE
    BIN_EDGE = args.bin_edge
    PROFILE_RANGE = args.profile_range
    PRECOND = {"auto": 0, "jacobi": 1, "multigrid": 2}[args.precond]
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "serve":
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
