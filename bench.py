#!/usr/bin/env python
"""Benchmark: quantized MLS-MPM particle-steps/s on one B300 (per GPU, replicas).

One "step" is one MLS-MPM time step of the whole scene on bit-packed fixed-point state
(P2G, grid update, G2P, dithered store, and the periodic tile re-sort), run by the
library's kernels on device-resident state.  Default workload: 3D fixed-corotated elastic
cubes, 16 x 512,000 = 8,192,000 particles, 256^3 grid, dt 5e-5 (synthetic scene:
seeded jittered cubes).  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank steps its own replica of the scene (independent seeds, no
collective on the data path): weak scaling, value = all particle-steps / max rank time.
"""
import argparse
import hashlib
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

METRIC = "quantized vs FP32 MPM particle-steps/s at rel err<=0.01; %HBM peak; p99 latency"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cubes3d", choices=["cubes3d", "dambreak3d", "block2d", "smoke"],
                    help="smoke: the quantized 2D smoke batch alone (its own JSON line)")
    ap.add_argument("--no-smoke", action="store_true", help="leave the smoke section out of the MPM line")
    ap.add_argument("--smoke-scenes", type=int, default=64)
    ap.add_argument("--smoke-fixed-scheme", action="store_true",
                    help="the smoke's eps 1e-3 scheme as written down instead of solved in the run")
    ap.add_argument("--no-smoke-validation", action="store_true", help="skip the smoke error-bound protocol")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--serving-duration", type=float, default=60.0,
                    help="seconds of Poisson arrivals in the serving run (0: skip it)")
    ap.add_argument("--fixed-scheme", action="store_true",
                    help="hand-written scheme instead of the solved one (quick runs)")
    ap.add_argument("--scheme-json", default=None,
                    help="load a scheme saved by --save-scheme instead of solving it again")
    ap.add_argument("--save-scheme", default=None, help="write the solved scheme to this file")
    ap.add_argument("--generic-kernel", action="store_true",
                    help="step with the library's step kernel instead of the one compiled for the scheme")
    ap.add_argument("--fp32-state", action="store_true",
                    help="time the FP32 state as the headline (the comparator's step kernel, for profiling)")
    ap.add_argument("--resolve-scheme", action="store_true",
                    help="solve the cubes' second-order scheme in this run instead of loading the cached one")
    ap.add_argument("--algorithm1-scheme", action="store_true",
                    help="the cubes' scheme from Algorithm 1 alone (no second-order refinement)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="fraction of the workload's cubes/columns (for quick runs only)")
    return ap.parse_args()


# ------------------------------------------------------------------------------ workloads
def solved_cubes_scheme(eps=0.01):
    """The cubes' scheme from the bit-allocation solve (Eq. 10) at relative error eps on
    the final particle positions, with sensitivities from the half-resolution scene."""
    from paper_2207_04658_b300 import autoquant
    scheme, rep = autoquant.cubes3d_scheme(eps)
    return scheme, rep


def workload(name, scale=1.0, seed_offset=0, scheme=None):
    from paper_2207_04658_b300 import scenes
    if name == "cubes3d":
        n_cubes = max(1, int(round(16 * scale)))
        # re-sort every 20 steps: the best period with margin over a 480-step run of this
        # workload with the scheme-specialised step kernel (ms per step, sort included:
        # 0.944 at 12, 0.933 at 16, 0.927 at 20, 0.922 at 24, 0.942 at 32, 1.247 at 48, where
        # particles have left their tiles)
        sc, s0 = scenes.cubes3d_scene(n_cubes=n_cubes, seed=2 + seed_offset, resort_every=20)
        sch = scheme if scheme is not None else scenes.fixed_scheme_3d("corotated")
        desc = {"workload": "3D fixed-corotated elastic cubes", "particles": int(s0.shape[0]),
                "cubes": n_cubes, "grid": "256^3", "dt": sc["dt"], "E": sc["E"], "nu": sc["nu"],
                "rho": sc["rho"], "ppc": 8, "initial_speed": 3.0,
                "scheme": {k: [f["bits"], f["frac"]] for k, f in sch.items()},
                "scheme_source": "qmpm_scheme_solve, eps 0.01 on final positions" if scheme is not None
                else "fixed", "resort_every": sc["resort_every"]}
    elif name == "dambreak3d":
        cells = max(8, int(round(256 * scale ** (1 / 3))))
        # re-sort every 64 steps: at dt 2e-5 the fluid moves ~0.03 cells a step, and a sweep
        # of the interval (8 ... 128, 2^27 particles) left the step kernel within 0.2 % while
        # the amortised sort (11.5 ms a pass) fell from 1.43 to 0.18 ms per step
        sc, s0 = scenes.dambreak3d_scene(column_cells=cells, seed=3 + seed_offset, resort_every=64)
        sch = scheme if scheme is not None else scenes.fixed_scheme_3d("fluid", C=(16, -2048.0, 2048.0))
        desc = {"workload": "3D weakly compressible dam break", "particles": int(s0.shape[0]),
                "grid": "512^3", "dt": sc["dt"], "bulk": sc["bulk"], "ppc": 8,
                "resort_every": sc["resort_every"],
                "scheme": {k: [f["bits"], f["frac"]] for k, f in sch.items()},
                "scheme_source": ("Algorithm 1, eps 0.01 on final positions, sensitivities of the column at "
                                  "quarter resolution" if scheme is not None else "fixed")}
    else:
        sc, s0 = scenes.block2d_scene(seed=1 + seed_offset)
        sch = scenes.block2d_scheme()
        desc = {"workload": "2D neo-Hookean block", "particles": int(s0.shape[0]), "grid": "128^2",
                "dt": sc["dt"], "resort_every": sc["resort_every"]}
    return sc, s0, sch, desc


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
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
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = [num(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------------------ our arm
def time_scene(qmpm, torch, sc, s0, sch, steps, warmup, dist_ctx, specialize=False):
    """K steps of one scene timed with CUDA events on its stream after `warmup` steps;
    specialize: step with the kernel compiled for the scheme at init (outside the timing)."""
    stream = torch.cuda.current_stream()
    g = qmpm.Scene(sc, sch, s0, stream=stream.cuda_stream, profile=True, specialize=specialize)
    for _ in range(warmup):
        g.step(1)
    torch.cuda.synchronize()
    g.profile(reset=True)
    dist_ctx.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        g.step(1)
    t1.record(stream)
    torch.cuda.synchronize()
    dist_ctx.barrier()
    ms = t0.elapsed_time(t1)
    prof = g.profile(reset=True)
    st = g.readback(state=False, ids=False)["stats"]
    return g, ms, prof, st


def e2e_scene(qmpm, torch, g, steps, warmup, chunks=0):
    """End to end through the host, every step: the packed state copied in from pinned host
    memory, the grid cleared and the P2G redone from it, the step, and the state copied back.
    Timed twice: through qmpm_step_host_stream (copies in `chunks` particle ranges, 0: the
    library's choice, one per 16 MiB of state up to 8; the download of a step's result
    overlapping the next step's upload), the headline, and
    through one qmpm_step_host call per step (the copies one after the other).  Returns
    (seconds pipelined, seconds one call per step, bytes each way per step)."""
    r = g.readback(state=False, words=True, ids=False)
    words = r["words"]
    hw = torch.from_numpy(words.copy()).pin_memory()
    qmpm.qmpm_step_host_stream(g.h, max(3, warmup), hw.data_ptr(), chunks)
    t = time.perf_counter()
    qmpm.qmpm_step_host_stream(g.h, steps, hw.data_ptr(), chunks)
    el_stream = time.perf_counter() - t
    hin = torch.from_numpy(hw.numpy().copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for _ in range(max(3, warmup)):
        qmpm.qmpm_step_host(g.h, 1, hin.data_ptr(), hout.data_ptr())
        hin, hout = hout, hin
    t = time.perf_counter()
    for _ in range(steps):
        qmpm.qmpm_step_host(g.h, 1, hin.data_ptr(), hout.data_ptr())
        hin, hout = hout, hin
    el = time.perf_counter() - t
    return el_stream, el, int(words.nbytes)


L2_BYTES = 126 * 2 ** 20  # B300 L2
STEP_SOURCES = ("step.cu", "step_kernels.cuh", "jit.cpp", "device_common.cuh", "mpm_device.cuh", "qmpm_internal.h")
SMOKE_SOURCES = ("smoke.cu", "device_common.cuh", "qmpm_internal.h")


def sources_sha256(names):
    """SHA-256 over the named csrc files in order: a committed counter record is used only
    while the kernel and every header it compiles from are unchanged since its capture."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2207_04658_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_counters(desc, n_particles, words=None):
    """DRAM bytes, warp instructions and thread instructions per launch of the step kernel
    from the committed ncu summary, scaled by the particle count to this workload; Nones
    when the kernel source changed since the capture."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "step_kernel_traffic*.json"))):
        try:
            rec = json.load(open(path))
            if rec.get("workload") != desc["workload"]:
                continue
            if rec.get("sources_sha256") != sources_sha256(STEP_SOURCES):
                return None, None, None
            if words is not None and rec.get("words_per_particle") not in (None, words):
                return None, None, None
            f = n_particles / rec["particles"]
            return (rec["dram_bytes_per_launch"] * f, rec["warp_instructions_per_launch"] * f,
                    rec.get("thread_instructions_per_launch", 0) * f or None)
        except Exception:
            return None, None, None
    return None, None, None


def issue_peak(peaks):
    """Warp-instruction issue peak: 148 SMs x 4 schedulers x 1 warp instruction per clock
    at the maximum SM clock."""
    mhz = peaks.get("sm_max_mhz", 2032.0)
    return 148 * 4 * mhz * 1e6


LANE_PEAK_SOURCE = "148 SMs x 4 schedulers x 32 lanes x 1 instruction/clk x max SM clock"


def alu_roofline(kernel, avg_ms, winst, tinst, peaks, **extra):
    """The issue-bound roofline of a kernel: the thread instructions it executes (the work
    its active lanes do) per second against 32 lanes x the warp-issue peak; the warp-issue
    rate (idle lanes of a warp count as issued) is reported beside it."""
    ipk = issue_peak(peaks)
    out = {"bound": "alu", "kernel": kernel, "avg_launch_ms": round(avg_ms, 5), "unit": "T lane-instructions/s",
           "peak": round(32 * ipk / 1e12, 3), "peak_source": LANE_PEAK_SOURCE}
    if tinst:
        ach = tinst / (avg_ms / 1e3)
        out.update({"achieved": round(ach / 1e12, 3), "frac": round(ach / (32 * ipk), 4),
                    "thread_instructions_per_launch": tinst})
    else:
        out.update({"achieved": None, "frac": None})
    if winst:
        w = winst / (avg_ms / 1e3)
        out["warp_issue"] = {"achieved": round(w / 1e9, 2), "peak": round(ipk / 1e9, 2),
                             "unit": "G warp-instructions/s", "frac": round(w / ipk, 4),
                             "warp_instructions_per_launch": winst}
    out.update(extra)
    return out


class _DevArray:
    """A raw device buffer seen by torch without a copy (__cuda_array_interface__)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


def device_positions(qmpm, torch, g):
    """Positions of a resident scene as a device tensor [N, dim] in initial particle order,
    decoded on the device (the packed words through qmpm_unpack_f32, FP32 words as they
    are); nothing crosses the host link."""
    w, ld, ids = qmpm.qmpm_state_device(g.h)
    N, nc, dim = g.N, g.n_comp, g.dim
    idx = torch.as_tensor(_DevArray(ids, N, "<i8"), device="cuda")
    if g.quantized:
        vals = torch.empty((N, nc), dtype=torch.float32, device="cuda")
        qmpm.qmpm_unpack_f32(dim, qmpm.MATERIALS[g.material], g._scheme_struct, w, N, ld, vals.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        pos = vals[:, :dim]
    else:
        planes = torch.as_tensor(_DevArray(w, nc * ld, "<f4"), device="cuda").view(nc, ld)
        pos = planes[:dim, :N].t()
    out = torch.empty((N, dim), dtype=torch.float32, device="cuda")
    out[idx] = pos
    torch.cuda.synchronize()
    return out


def dambreak_variants(qmpm, torch, args, dc, peaks):
    """The dam break as the scaling experiment states it (Sec. 8.3): Algorithm 1's schemes at
    relative error bounds 0.1 and 0.01 on the final positions (sensitivities and ranges of the
    column at quarter resolution), each with dithered and with round-to-nearest stores, timed
    like the headline and run for the scene's full step count against the FP32 run of the
    same kernels (z and RMS position error, compared on the device).  Returns the variants
    and the scheme of the headline (eps 0.01, dithered)."""
    from paper_2207_04658_b300 import autoquant
    schemes, info = autoquant.dambreak3d_schemes((0.1, 0.01))
    sc, s0, _, desc = workload("dambreak3d", args.scale, seed_offset=dc.rank)
    T = int(sc["steps"])
    g32 = qmpm.Scene(sc, None, s0)
    g32.step(T)
    x32 = device_positions(qmpm, torch, g32)
    z32 = float((x32.double() ** 2).sum(1).mean())
    rms = float(torch.sqrt((x32.double() ** 2).sum(1).mean()))
    g32.close()
    out = []
    for eps in (0.1, 0.01):
        scheme, res = schemes[eps]
        for dither in (True, False):
            s = dict(sc, dither=dither)
            k = max(8, min(args.steps, 64))
            g, ms, prof, st = time_scene(qmpm, torch, s, s0, scheme, k, args.warmup, dc,
                                         specialize=not args.generic_kernel)
            W = g.n_words
            g.close()
            gq = qmpm.Scene(s, scheme, s0, stats=True, specialize=not args.generic_kernel)
            gq.step(T)
            xq = device_positions(qmpm, torch, gq)
            sat = gq.readback(state=False, ids=False)["stats"]["saturations"]
            gq.close()
            d = (xq.double() - x32.double())
            err = float(torch.sqrt((d ** 2).sum(1).mean())) / rms
            zq = float((xq.double() ** 2).sum(1).mean())
            del xq, d
            names = ("x", "v", "C", "J")
            out.append({"eps": eps, "dither": dither, "bits": [scheme[n]["bits"] for n in names],
                        "frac": [scheme[n]["frac"] for n in names], "solved_bits": res["bits"],
                        "words_per_particle": W, "bytes_per_particle": 4 * W,
                        "value": dc.world * s0.shape[0] * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k,
                        "timed_steps": k,
                        "step_kernel_ms": round(prof["step_ms"] / max(1, prof["step_launches"]), 4),
                        "accuracy": {"steps": T, "z_rel_err": abs(zq - z32) / abs(z32), "rms_pos_err_rel": err,
                                     "saturations": sat, "within_eps": err <= eps, "within_3eps": err <= 3 * eps,
                                     "reference": "FP32 run of the same kernels (an FP64 oracle run of 2^27 "
                                                  "particles is out of reach on the host; the reduced case is "
                                                  "checked against the FP64 oracle in tests/test_gpu_dambreak.py)"}})
            torch.cuda.empty_cache()
    return out, schemes[0.01][0], info


def accuracy(qmpm, sc, s0, sch, specialize=False):
    """Full rollouts (the scene's step count) of the quantized and the FP32 state from the
    same initial state: relative error of z = mean |x|^2 and RMS per-particle position
    error over RMS position (the bound the scheme was solved for), compared on the device.
    specialize: the quantized run steps with the kernel compiled for the scheme, as timed."""
    import torch
    steps = int(sc.get("steps", 1000))
    out = {}
    for name, scheme in (("quant", sch), ("fp32", None)):
        g = qmpm.Scene(sc, scheme, s0, stats=True, specialize=specialize)
        g.step(steps)
        out[name] = (device_positions(qmpm, torch, g).double(), g.readback(state=False, ids=False)["stats"])
        g.close()
    xq, xf = out["quant"][0], out["fp32"][0]
    zq, zf = float((xq ** 2).sum(1).mean()), float((xf ** 2).sum(1).mean())
    rms_err = float(torch.sqrt(((xq - xf) ** 2).sum(1).mean()))
    rms_pos = float(torch.sqrt((xf ** 2).sum(1).mean()))
    return {"steps": steps, "z_quant": zq, "z_fp32": zf, "z_rel_err": abs(zq - zf) / abs(zf),
            "rms_pos_err_rel": rms_err / rms_pos, "saturations": out["quant"][1]["saturations"],
            "reference": "FP32 run of the same kernels (the FP64 oracle comparison at this size is in "
                         "tests/test_gpu_rollout_reference.py)"}


def latency_spread(lat, windows=3, resamples=1000, seed=7):
    """Run-to-run spread of the latency percentiles: p50 and p99 of consecutive windows of
    the arrivals (each its own run), and a bootstrap 90 % interval of each over requests."""
    if len(lat) < 10:
        return None
    gen = np.random.default_rng(seed)
    boot = np.percentile(gen.choice(lat, (resamples, len(lat))), [50, 99], axis=1)
    parts = np.array_split(lat, windows)
    return {"windows": [{"p50_ms": round(float(np.percentile(w, 50)), 2),
                         "p99_ms": round(float(np.percentile(w, 99)), 2), "requests": int(len(w))} for w in parts],
            "bootstrap90_p50_ms": [round(float(v), 2) for v in np.percentile(boot[0], [5, 95])],
            "bootstrap90_p99_ms": [round(float(v), 2) for v in np.percentile(boot[1], [5, 95])]}


def serving(qmpm, duration, rate=20.0, budget_gb=120.0, max_active=64, dc=None):
    """The serving workload: Poisson arrivals of scenes (2D/3D x elastic/fluid, particle
    counts log-uniform in [1e4, 4e6], grids 64^3..256^3 or 128^2..1024^2, schemes solved at
    eps 0.1 or 0.01, 200 steps) submitted to the engine at their arrival times; rollout
    latency (submit to finished, measured) percentiles and aggregate particle-steps/s."""
    from paper_2207_04658_b300 import autoquant, scenes
    t_solve = time.perf_counter()
    schemes = autoquant.serving_schemes()
    t_solve = time.perf_counter() - t_solve
    from paper_2207_04658_b300.replicas import shard
    reqs = scenes.serving_requests(rate=rate, duration=duration, seed=5)
    if dc is not None and dc.world > 1:
        reqs = shard(reqs, dc.rank, dc.world)  # replicas: each GPU serves every world-th request
    # the scenes are drawn ahead of their arrival times by a pool of threads (numpy releases
    # the GIL) with a bounded lookahead, and submitted without a copy at their arrival times;
    # finished requests are polled as they come, which releases their borrowed states
    import collections
    import concurrent.futures as cf

    def draw(r):
        return scenes.serving_scene(r["dim"], r["material"], r["n"], r["grid_log2"], r["seed"])

    lookahead = 48
    ex = cf.ThreadPoolExecutor(8)
    pending = collections.deque(ex.submit(draw, r) for r in reqs[:lookahead])
    t_gen = time.perf_counter()
    for f in list(pending)[:16]:  # a head start before the clock starts
        f.result()
    t_gen = time.perf_counter() - t_gen
    eng = qmpm.Engine(budget_bytes=int(budget_gb * 2 ** 30), resort_every=8, max_active=max_active)
    eng.start()
    t0 = time.perf_counter()
    lateness = []
    submitted = 0
    particle_steps = 0
    recs = []
    for i, r in enumerate(reqs):
        sc, s0 = pending.popleft().result()
        if i + lookahead < len(reqs):
            pending.append(ex.submit(draw, reqs[i + lookahead]))
        wait = r["t"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        lateness.append(max(0.0, -wait))
        eng.submit(sc, schemes[(r["dim"], r["material"], r["grid_log2"], r["eps"])], s0, sc["steps"], borrow=True)
        submitted += 1
        particle_steps += s0.shape[0] * sc["steps"]
        if i % 16 == 15:
            recs += eng.poll(max_n=256)
    ex.shutdown()
    eng.stop(drain=True)
    recs += eng.poll(max_n=max(1, submitted))
    st = eng.stats()
    eng.close()
    done = [r for r in recs if r["status"] == qmpm.REQ_DONE]
    lat = np.array([r["t_done"] - r["t_submit"] for r in done]) * 1e3
    span = max(r["t_done"] for r in done) - min(r["t_submit"] for r in done) if done else float("nan")
    if dc is not None and dc.world > 1:
        import torch
        # whole job: particle-steps of all ranks over the longest rank's span; the worst p99
        ps = dc.sum(torch, st["particle_steps"])
        span = dc.max(torch, span)
        st["particle_steps"] = ps
        p99_all = dc.max(torch, float(np.percentile(lat, 99)) if len(lat) else 0.0)
    else:
        p99_all = float(np.percentile(lat, 99)) if len(lat) else None
    return {"p99_ms_all_ranks": round(p99_all, 2) if p99_all is not None else None,"requests": submitted, "done": len(done), "failed": len(recs) - len(done),
            "arrival_rate_per_s": rate, "duration_s": duration,
            "p50_ms": round(float(np.percentile(lat, 50)), 2) if len(lat) else None,
            "p99_ms": round(float(np.percentile(lat, 99)), 2) if len(lat) else None,
            "p99_requests_above": int(np.sum(lat > np.percentile(lat, 99))) if len(lat) else None,
            "spread": latency_spread(lat),
            "mean_ms": round(float(lat.mean()), 2) if len(lat) else None,
            "particle_steps_per_s": st["particle_steps"] / span if done else None, "unit": UNIT,
            "particle_steps": st["particle_steps"], "offered_particle_steps": particle_steps,
            "budget_gb": budget_gb, "max_active": max_active, "iterations": st["iterations"],
            "graph_launches": st["graph_launches"], "kernel_launches": st["kernel_launches"],
            "submit_lateness_p99_ms": round(float(np.percentile(lateness, 99)) * 1e3, 2) if lateness else None,
            "scheme_solve_s": round(t_solve, 2), "scene_generation_s": round(t_gen, 2),
            "mix": "uniform over 2D neo-Hookean, 2D fluid, 3D fixed-corotated, 3D fluid; N log-uniform "
                   "[1e4, 4e6]; eps uniform {0.1, 0.01}; 200 steps; schemes from Algorithm 1 per class and grid"}


def host_cpu():
    """The host's CPU model, its logical cores (those this process may run on) and memory."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    try:
        mem = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        mem = 0
    return {"model": model, "cores": cores, "logical_cpus": os.cpu_count(), "mem_available_gb": round(mem / 2 ** 30, 1)}


def _oracle_slice(job):
    """One oracle process of the aggregate: its slice of the workload's initial state (read
    from the shared .npy file), `steps` quantized steps on the full grid."""
    sc, sch, path, lo, hi, steps = job
    import oracle
    s0 = np.array(np.load(path, mmap_mode="r")[lo:hi])
    ro = oracle.QuantRollout(sc, sch, s0)
    t = time.perf_counter()
    ro.step(steps)
    return (hi - lo) * steps, time.perf_counter() - t


def cpu_baseline(name, scheme=None, sample_steps=2):
    """The oracle (single-threaded FP64 C, as it stands) on bounded samples of the same
    workload and scheme.  Single core: the first cube (or a slice of the column) on the full
    grid, `sample_steps` quantized steps (more for small scenes).  Aggregate: one oracle process per host core (capped
    by the memory each needs: the full FP64 grid plus its slice), each stepping a disjoint
    slice of the whole scene; value = the particle-steps of all processes over the slowest
    one's time.  The unquantized FP64 oracle step on the single-core sample is reported
    beside it."""
    import multiprocessing as mp
    import oracle
    sc, s0, sch, desc = workload(name, scheme=scheme)
    n = {"cubes3d": 512_000, "dambreak3d": 256_000}.get(name, s0.shape[0])
    what = {"cubes3d": "first cube of 16", "dambreak3d": "first particles of the column"}.get(name, "whole scene")
    # small scenes take more steps, so that every sample is ~1e6 particle-steps or more
    steps1 = max(sample_steps, min(100, int(2e6 // n)))
    ro = oracle.QuantRollout(sc, sch, s0[:n])
    t = time.perf_counter()
    ro.step(steps1)
    el = time.perf_counter() - t
    one = n * steps1 / el
    rf = oracle.Fp64Rollout(sc, s0[:n])
    t = time.perf_counter()
    rf.step(steps1)
    one_fp64 = n * steps1 / (time.perf_counter() - t)
    del rf
    host = host_cpu()
    grid_bytes = oracle.n_nodes(ro.ph) * (1 + ro.ph.dim) * 8
    del ro
    per_proc = 2 * grid_bytes + 3 * 8 * s0.shape[1] * (s0.shape[0] // max(1, host["cores"]))
    P = max(1, min(host["cores"], 256, int(0.6 * host["mem_available_gb"] * 2 ** 30 // max(1, per_proc))))
    out = {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{what} ({n} particles) on the full grid, {steps1} steps, the bench's scheme",
           "host": host, "single_core": one, "single_core_fp64_unquantized": one_fp64}
    N = s0.shape[0]
    if P > 1:
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "s0.npy")
            np.save(path, s0)
            del s0
            bounds = [N * i // P for i in range(P + 1)]
            steps_p = max(1, min(100, int(2e6 // max(1, N // P))))
            jobs = [(sc, sch, path, bounds[i], bounds[i + 1], steps_p) for i in range(P)]
            with mp.get_context("spawn").Pool(P) as pool:
                res = pool.map(_oracle_slice, jobs, chunksize=1)
        work = sum(r[0] for r in res)
        out.update(value=work / max(r[1] for r in res), cores=P,
                   sample=f"{P} oracle processes (one per core, memory permitting), each a disjoint "
                          f"1/{P} of the whole {N}-particle scene on the full grid for {steps_p} quantized "
                          f"step{'s' if steps_p > 1 else ''}, "
                          "the bench's scheme; value = all particle-steps over the slowest process's time")
    return out


# ------------------------------------------------------------------------------ smoke
SMOKE_METRIC = "quantized 2D smoke cell-steps/s (advection-reflection, 64 Jacobi sweeps per projection)"
SMOKE_UNIT = "cell-steps/s"
SMOKE_FIXED_SCHEME = {"v": dict(bits=13, frac=10, offset=-3616), "p": dict(bits=14, frac=18, offset=-4288)}


def smoke_counters():
    """Warp instructions and DRAM bytes per Jacobi launch from the committed ncu summary,
    or (None, None) when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "smoke_jacobi_counters.json")
    if not os.path.exists(path):
        return None, None, None
    try:
        rec = json.load(open(path))
        if rec.get("sources_sha256") != sources_sha256(SMOKE_SOURCES):
            return None, None, None
        return rec["warp_instructions_per_launch"], rec["dram_bytes_per_launch"], rec
    except Exception:
        return None, None, None


def smoke_section(args, peaks, dc, torch):
    """The quantized smoke batch (Sec. 8.1's 2D advection-reflection workload): S scenes of
    the 256^2 plume stepped together by one CUDA graph per step; the scheme Algorithm 1
    solves at eps 1e-3 from noise-injection sensitivities.  Device-timed throughput
    (quantized and FP32), the Jacobi kernel against the issue peak, an end-to-end rollout
    from host state, and the error-bound protocol at eps 1e-2 and 1e-3 (20 dither seeds)."""
    from paper_2207_04658_b300 import scenes, smoke
    sc = scenes.smoke_scene()
    T = sc["steps"]
    S = args.smoke_scenes
    n = sc["n"]
    if args.smoke_fixed_scheme:
        scheme = SMOKE_FIXED_SCHEME
        source = "written down: the bias-aware solve's eps 1e-3 result on this scene (bits 13/14, frac 10/18)"
    else:
        scheme, rep = smoke.solve(sc, T, 1e-3, bias_aware=True)
        source = ("qmpm_scheme_solve at eps 1e-3 on z = sum d^2 after 100 steps, noise-injection "
                  "sensitivities (32 antithetic pairs per type), bits added for the second-order bias")
    steps = max(10, min(args.steps, 200))
    warm = max(3, args.warmup)
    st = torch.cuda.Stream()
    out = {"config": {"workload": "2D smoke plume batch", "scenes": S, "grid": f"{n}^2", "jacobi": sc["jacobi"],
                      "dt": sc["dt"], "rollout_steps": T, "scheme": scheme,
                      "scheme_source": source,
                      "l2": "L2-resident working set (packed state "
                            f"{S * (2 * n * (n + 1) * scheme['v']['bits'] / 8 + 4 * n * n) / 1e6:.0f} MB)"}}
    for name, sch in (("quant", scheme), ("fp32", None)):
        with smoke.Smoke(sc, sch, S, seeds=list(range(S)), stream=st.cuda_stream) as g:
            g.step(warm)
            torch.cuda.synchronize()
            dc.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            g.step(steps)
            e1.record(st)
            torch.cuda.synchronize()
            ms = dc.max(torch, e0.elapsed_time(e1))
            info = g.info()
        out[name] = {"value": dc.world * S * n * n * steps / (ms / 1e3), "unit": SMOKE_UNIT,
                     "ms_per_step": ms / steps, "state_bytes_per_scene": info["state_bytes"],
                     "launches_per_step": info["launches_per_step"]}
    out["value"] = out["quant"]["value"]
    out["quantized_over_fp32"] = round(out["quant"]["value"] / out["fp32"]["value"], 4)
    out["gpu_launches"] = out["quant"]["launches_per_step"] * steps
    # the Jacobi sweeps, timed by events around their launches
    with smoke.Smoke(dict(sc, profile=True), scheme, S, seeds=list(range(S)), stream=st.cuda_stream) as g:
        g.step(warm)
        g.profile()
        g.step(steps)
        prof = g.profile()
    jac_ms = prof["jacobi_ms"] / max(1, prof["jacobi_launches"])
    winst, dram, rec = smoke_counters()
    f = S / rec["scenes"] if (winst is not None and rec.get("n") == n) else None
    out["roofline"] = alu_roofline("jacobi_kernel (4 dithered pressure sweeps per launch, shared-memory tiles)",
                                   jac_ms, winst * f if f else None,
                                   rec.get("thread_instructions_per_launch", 0) * f if f else None, peaks,
                                   share_of_step=round(prof["jacobi_ms"] / prof["step_ms"], 3),
                                   traffic=dram * f if f else None)
    # end to end: every step the whole batch's state from pinned host arrays, one step, the
    # state and z back to the host (the batch transfer calls; FP32 arrays both ways)
    pin = lambda *shape: torch.zeros(shape, dtype=torch.float32).pin_memory()  # noqa: E731
    hu, hv, hd = pin(S, n, n + 1), pin(S, n + 1, n), pin(S, n, n)
    with smoke.Smoke(sc, scheme, S, seeds=list(range(S)), stream=st.cuda_stream) as g:
        g.step(max(warm, 20))
        g.get_states(hu, hv, hd)  # a developed plume
        k = max(3, min(steps, 20))
        g.set_states(hu, hv, hd)
        g.step(1)
        g.get_states(hu, hv, hd)
        t = time.perf_counter()
        for _ in range(k):
            g.set_states(hu, hv, hd)
            g.step(1)
            g.get_states(hu, hv, hd)
            g.measure()
        el = dc.max(torch, time.perf_counter() - t)
    nbytes = 4 * (hu.numel() + hv.numel() + hd.numel())
    out["e2e"] = {"value": dc.world * S * n * n * k / el, "unit": SMOKE_UNIT, "h2d_bytes_per_step": nbytes,
                  "d2h_bytes_per_step": nbytes + 8 * S,
                  "path": "qmpm_smoke_set_states from pinned host arrays, one step of the batch, "
                          "qmpm_smoke_get_states and z back, every step"}
    if dc.rank == 0 and not args.no_smoke_validation:
        res = smoke.error_bound_protocol(sc, T, [1e-2, 1e-3], runs=20)
        out["error_bound"] = [{k: r[k] for k in ("eps", "solve", "bits", "frac", "pred_sigma_dither", "pred_bias",
                                                 "obs_rms", "bias", "z_std", "success_3eps", "compression")}
                              for r in res["results"]]
        out["error_bound_z_ref"] = res["z_ref"]
    return out


def smoke_cpu_baseline(steps=3):
    """The smoke oracle (single-threaded FP64 C, quantized stores) on one 256^2 scene."""
    import oracle
    from paper_2207_04658_b300 import scenes
    sc = scenes.smoke_scene()
    sch = {"v": dict(bits=16, frac=12, offset=-(1 << 15)), "p": dict(bits=16, frac=18, offset=-(1 << 15))}
    ro = oracle.SmokeRollout(sc, sch)
    t = time.perf_counter()
    ro.step(steps)
    el = time.perf_counter() - t
    return {"value": sc["n"] ** 2 * steps / el, "unit": SMOKE_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one 256^2 scene of the batch, {steps} quantized steps"}


def run_smoke(args):
    import torch
    from paper_2207_04658_b300 import build
    build.build()
    dc = DistCtx()
    dc.init(torch)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    clocks = ClockSampler(dc.local)
    clocks.start()
    sm = smoke_section(args, peaks, dc, torch)
    clk = clocks.stop()
    line = {"metric": SMOKE_METRIC, "value": sm["value"], "unit": SMOKE_UNIT, "n_gpus": dc.world,
            "steps": max(10, min(args.steps, 200)), "warmup": max(3, args.warmup),
            "ms_per_step": sm["quant"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "gpu_launches": sm["gpu_launches"],
            "config": dict(sm["config"], parallelism=f"replicas{dc.world}"), "roofline": sm["roofline"],
            "clocks": clk, "e2e": sm["e2e"], "fp32": sm["fp32"], "quantized_over_fp32": sm["quantized_over_fp32"]}
    if "error_bound" in sm:
        line["error_bound"] = sm["error_bound"]
    if dc.rank == 0 and dc.world == 1 and not args.no_cpu:
        line["cpu_baseline"] = smoke_cpu_baseline()
    if dc.rank == 0:
        print(json.dumps(line), flush=True)
    dc.close()


def DistCtx():
    from paper_2207_04658_b300.replicas import Replicas
    return Replicas()


def run_ours(args):
    import torch
    from paper_2207_04658_b300 import build, qmpm
    build.build()
    dc = DistCtx()
    dc.init(torch)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    peak_note = "of measured" if "hbm_gbs" in peaks else "of fallback"

    solve_info = None
    scheme = None
    if args.scheme_json:
        with open(args.scheme_json) as f:
            saved = json.load(f)
        scheme, solve_info = saved["scheme"], saved["solve"]
    elif args.workload == "cubes3d" and not args.fixed_scheme:
        from paper_2207_04658_b300 import autoquant
        cached = None if (args.resolve_scheme or args.algorithm1_scheme) else autoquant.load_cubes3d_scheme(0.01)
        if cached is not None or args.resolve_scheme:
            if cached is None:
                scheme, rep = autoquant.cubes3d_second_order_scheme(0.01)
                rep = autoquant._summary(rep)
            else:
                scheme, rep = cached["scheme"], cached["report"]
            last = rep["rounds"][-1]
            solve_info = {"bits": {k: v["bits"] for k, v in scheme.items()},
                          "frac": {k: v["frac"] for k, v in scheme.items()},
                          "algorithm1_bits": {k: v["bits"] for k, v in rep["algorithm1"].items()},
                          "pred_bias": last["pred_bias"], "pred_var": last["pred_var"],
                          "bound": (0.01 * rep["z"]) ** 2, "rounds": len(rep["rounds"]),
                          "source": ("cached: python -m paper_2207_04658_b300.autoquant cubes3d --eps 0.01"
                                     if cached is not None else "solved in this run"),
                          "method": "Algorithm 1 (sensitivities of the 16 cubes at half resolution), refined "
                                    "with the second-order term (noise injection at full resolution), the last "
                                    "word's free bits spent on wider windows, accepted by quantized rollouts "
                                    "against the FP32 rollout at full resolution"}
            acc = rep.get("acceptance") or []
            if acc:
                solve_info["acceptance"] = {"rounds": len(acc), "rel_err": acc[-1]["rel_err"],
                                            "saturations": acc[-1]["saturations"],
                                            "dither_seeds": acc[-1].get("seeds")}
        else:
            scheme, rep = solved_cubes_scheme(0.01)
            solve_info = {"bits": rep["solve"]["bits"], "frac": rep["solve"]["frac"],
                          "pred_err": rep["solve"]["pred_err"],
                          "bound": (0.01 * rep["sensitivities"]["z"]) ** 2,
                          "method": "Algorithm 1 alone",
                          "sensitivity_run": "16 cubes at half resolution (1,024,000 particles, 128^3), "
                                             "1000 steps, 2 Gaussian seeds on x_T"}
    variants = None
    if args.workload == "dambreak3d" and not args.fixed_scheme and not args.scheme_json:
        variants, scheme, dinfo = dambreak_variants(qmpm, torch, args, dc, peaks)
        solve_info = {"method": "Algorithm 1 (the scaling procedure of Sec. 8.3)", "eps": 0.01,
                      "sensitivity_run": "column of 64^3 cells on a 128^3 grid (2,097,152 particles), 500 steps, "
                                         "2 Gaussian seeds on x_T",
                      "bits": {k: v["bits"] for k, v in scheme.items()}}
    if args.save_scheme and scheme is not None and dc.rank == 0:
        with open(args.save_scheme, "w") as f:
            json.dump({"scheme": scheme, "solve": solve_info}, f)
    sc, s0, sch, desc = workload(args.workload, args.scale, seed_offset=dc.rank, scheme=scheme)
    if args.fp32_state:  # the comparator alone (profiling the FP32 step kernel)
        sch = None
        desc = dict(desc, scheme=None, scheme_source="FP32 state")
    N = s0.shape[0]
    clocks = ClockSampler(dc.local)
    clocks.start()
    spec = not args.generic_kernel
    g, ms, prof, st = time_scene(qmpm, torch, sc, s0, sch, args.steps, args.warmup, dc, specialize=spec)
    clk = clocks.stop()
    kinfo = qmpm.qmpm_step_kernel_info(g.h)
    ms_max = dc.max(torch, ms)
    W = g.n_words
    from paper_2207_04658_b300.replicas import job_throughput
    value = job_throughput(N * args.steps, dc.world, ms_max / 1e3)

    # dominant kernel: the fused step kernel
    step_avg_ms = prof["step_ms"] / max(1, prof["step_launches"])
    node_bytes = 16
    nodes = st["active_blocks"] * (64 if sc["dim"] == 3 else 16)
    alg_bytes = N * 2 * 4 * W + nodes * 2 * node_bytes
    achieved = alg_bytes / (step_avg_ms / 1e3) / 1e9
    traffic, winst, tinst = kernel_counters(desc, N, W)
    hbm = {"achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(achieved / hbm_peak, 4), "peak_source": peak_note,
           "alg_bytes_per_launch": alg_bytes}
    if winst is not None:
        # the step kernel is issue bound (see profiles/): report against the issue peak
        roofline = alu_roofline("step_kernel (G2P -> dithered store -> P2G)", step_avg_ms, winst, tinst, peaks,
                                traffic=traffic, hbm=hbm)
    else:
        roofline = dict({"bound": "hbm", "traffic": None,
                         "kernel": "step_kernel (G2P -> dithered store -> P2G)",
                         "avg_launch_ms": round(step_avg_ms, 4)}, **hbm)
    breakdown = {"step_ms_per_step": round(prof["step_ms"] / args.steps, 4),
                 "clear_ms_per_step": round(prof["clear_ms"] / args.steps, 4),
                 "sort_ms_per_step": round(prof["sort_ms"] / args.steps, 4),
                 "launch_gap_ms_per_step": round((ms - prof["step_ms"] - prof["clear_ms"]
                                                  - prof["sort_ms"]) / args.steps, 4)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dc.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "gpu_launches": int(prof["kernel_launches"]),
            "config": dict(desc, replicas=dc.world, l2=(f"inputs larger than L2 (packed state {N * 4 * W / 1e6:.0f} MB "
                           "per replica, two buffers plus the grid)" if 2 * N * 4 * W > L2_BYTES else
                           f"L2-resident, not flushed (packed state {N * 4 * W / 1e6:.1f} MB): a latency "
                           "measurement, not a bandwidth one"),
                           bytes_per_particle_quantized=4 * W, bytes_per_particle_fp32=4 * g.n_comp,
                           compression=round(g.n_comp / W, 3), parallelism=f"replicas{dc.world}"),
            "roofline": roofline, "breakdown": breakdown, "clocks": clk,
            "step_kernel": {"specialized_to_the_scheme": kinfo["specialized"],
                            "compile_seconds": round(kinfo["compile_seconds"], 3),
                            "how": ("the library's step kernel source compiled at qmpm_init (NVRTC, sm_103a) with "
                                    "the scheme's codec table as constants, outside the timed region"
                                    if kinfo["specialized"] else "the step kernel compiled with the library")},
            "stats": {"active_blocks": st["active_blocks"], "out_of_tile": st["out_of_tile"]}}
    if not args.no_e2e:
        k = max(3, min(args.steps // 4, 50))
        el, el_serial, nbytes = e2e_scene(qmpm, torch, g, k, 3)
        el, el_serial = dc.max(torch, el), dc.max(torch, el_serial)
        line["e2e"] = {"value": dc.world * N * k / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes,
                       "path": "qmpm_step_host_stream: pinned host words -> device, P2G, step, -> host, every "
                               "step, copies in up to 8 particle ranges (download of one overlapping upload of the next)",
                       "one_call_per_step": {"value": dc.world * N * k / el_serial, "unit": UNIT,
                                             "path": "qmpm_step_host, copies one after the other"}}
    g.close()
    if kinfo["specialized"]:
        # the same steps with the library's step kernel, for comparison
        gg, msg, profg, _ = time_scene(qmpm, torch, sc, s0, sch, args.steps, args.warmup, dc)
        gg.close()
        msg = dc.max(torch, msg)
        line["step_kernel"]["library_kernel"] = {
            "value": dc.world * N * args.steps / (msg / 1e3), "unit": UNIT, "ms_per_step": msg / args.steps,
            "step_kernel_ms": round(profg["step_ms"] / max(1, profg["step_launches"]), 4)}
    if not args.no_fp32:
        g32, ms32, prof32, st32 = time_scene(qmpm, torch, sc, s0, None, args.steps, args.warmup, dc,
                                             specialize=spec)
        ms32 = dc.max(torch, ms32)
        v32 = dc.world * N * args.steps / (ms32 / 1e3)
        s32 = prof32["step_ms"] / max(1, prof32["step_launches"])
        alg32 = N * 2 * 4 * g32.n_words + st32["active_blocks"] * (64 if sc["dim"] == 3 else 16) * 32
        line["fp32"] = {"value": v32, "unit": UNIT, "ms_per_step": ms32 / args.steps,
                        "step_kernel_ms": round(s32, 4),
                        "step_kernel_gbs": round(alg32 / (s32 / 1e3) / 1e9, 1),
                        "quantized_over_fp32": round(value / v32, 4),
                        "step_kernel": ("compiled at qmpm_init with the record's 24-word count as a constant, as the "
                                        "quantized kernel" if spec else "the step kernel compiled with the library")}
        if spec:
            gl, msl, profl, _ = time_scene(qmpm, torch, sc, s0, None, args.steps, args.warmup, dc)
            gl.close()
            msl = dc.max(torch, msl)
            line["fp32"]["library_kernel"] = {
                "value": dc.world * N * args.steps / (msl / 1e3), "unit": UNIT, "ms_per_step": msl / args.steps,
                "step_kernel_ms": round(profl["step_ms"] / max(1, profl["step_launches"]), 4)}
        if not args.no_e2e:
            # the same end-to-end path on FP32 state: four times the bytes over the host link
            k = max(3, min(args.steps // 4, 50))
            el32, el32_serial, nb32 = e2e_scene(qmpm, torch, g32, k, 3)
            el32, el32_serial = dc.max(torch, el32), dc.max(torch, el32_serial)
            line["fp32"]["e2e"] = {"value": dc.world * N * k / el32, "unit": UNIT,
                                   "h2d_bytes_per_step": nb32, "d2h_bytes_per_step": nb32,
                                   "one_call_per_step": dc.world * N * k / el32_serial}
            if "e2e" in line:
                line["e2e"]["quantized_over_fp32"] = round(line["e2e"]["value"] / line["fp32"]["e2e"]["value"], 3)
        g32.close()
    if solve_info is not None:
        line["scheme_solve"] = solve_info
    if variants is not None:
        line["variants"] = variants
    if not args.no_accuracy and dc.rank == 0 and variants is None:
        line["accuracy"] = accuracy(qmpm, sc, s0, sch, specialize=spec)
    if args.serving_duration > 0:
        line["serving"] = serving(qmpm, args.serving_duration, dc=dc)
    if not args.no_smoke:
        line["smoke"] = smoke_section(args, peaks, dc, torch)
    if dc.rank == 0 and dc.world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.workload, scheme=scheme)
    if dc.rank == 0:
        print(json.dumps(line), flush=True)
    dc.close()


def run_reference(args):
    """The reference arm: the CPU oracle (single-threaded FP64 C, as it stands) on a
    bounded sample of the same workload, each step one quantized oracle step."""
    dc = DistCtx()
    if dc.rank != 0:
        return
    if args.workload == "smoke":
        b = smoke_cpu_baseline(max(1, min(args.steps, 20)))
        line = {"impl": "reference", "metric": SMOKE_METRIC, "value": b["value"], "unit": SMOKE_UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 256 * 256 / b["value"] * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "2D smoke plume batch", "grid": "256^2", "jacobi": 64},
                "cpu_baseline": b, "e2e": {"value": b["value"], "unit": SMOKE_UNIT, "h2d_bytes_per_step": 0,
                                           "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import oracle
    scheme = None
    if args.workload == "cubes3d" and not args.fixed_scheme:
        # our arm's scheme: the cached second-order scheme (solving it needs a device)
        from paper_2207_04658_b300 import autoquant
        cached = autoquant.load_cubes3d_scheme(0.01)
        scheme = cached["scheme"] if cached is not None else None
    sc, s0, sch, desc = workload(args.workload, args.scale, scheme=scheme)
    if scheme is not None:
        desc = dict(desc, scheme_source="cached: python -m paper_2207_04658_b300.autoquant cubes3d --eps 0.01 "
                                        "(the scheme the GPU arm times)")
    n = {"cubes3d": 64_000, "dambreak3d": 64_000}.get(args.workload, s0.shape[0])
    sample = f"first {n} particles of the scene on its full grid, one quantized oracle step per step"
    ro = oracle.QuantRollout(sc, sch, s0[:n])
    ro.step(args.warmup)
    t = time.perf_counter()
    ro.step(args.steps)
    el = time.perf_counter() - t
    v = n * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "smoke":
        run_smoke(a)
    else:
        run_ours(a)
