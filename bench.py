#!/usr/bin/env python
"""Benchmark of the first-order MCPT(2) dimer term on one GB300.

Workload (default): lattice-10x10x10-cheb2 -- 1000 monomers of 32 AO / 5
occupied on a 3.0 A cubic lattice, all 42,092 dimers with Chebyshev distance
<= 2, 706 GB of FP64 integral blocks (2 x 32^4 per dimer), more than the
device holds.  They run in waves through one context: each wave's blocks are
generated on the device (untimed), then one step = one wave (~2,300 dimers,
36 GB, far above the 129 MB L2) through the whole path -- the first half (the
AO-reading transform), the second half with FP64 denominators and energies,
and the per-monomer accumulation -- in the BF16x2 form unless --precision
says otherwise.  The line carries the full-lattice error against the stored
oracle values, the FP64 form on the same waves, the CPU oracle on a sample
and an end-to-end leg through the C ABI from pinned host buffers.
--workload lattice-5x5x5-cheb1 (resident, 1036 dimers) and the other
workloads run the same path.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

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

METRIC = "dimer energies/sec"
UNIT = "dimers/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="bf16x2", choices=["tf32", "bf16x3", "bf16x2", "fp32c", "fp64", "fp64e"])
    p.add_argument("--workload", default="lattice-10x10x10-cheb2")
    p.add_argument("--wave-gb", type=float, default=WAVE_BUDGET / (1 << 30),
                   help="streamed workloads: GiB of integral blocks per wave (one wave = one step)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--fp64-epilogue", action="store_true",
                   help="mixed forms: energy epilogue on the FP64 pipe instead of FP32 pairs (for comparison)")
    p.add_argument("--tune", type=int, default=1, help="streamed workloads: autotune each wave's launch choices (1/0)")
    p.add_argument("--max-waves", type=int, default=64,
                   help="streamed workloads with more waves run only the waves the steps cover")
    p.add_argument("--cpu-sample", type=int, default=1024, help="dimers in the oracle's timed sample (at most)")
    p.add_argument("--no-extras", action="store_true",
                   help="report none of the extras (coupling, td2, df, FP64 form, FP64E form, e2e, CPU baseline)")
    p.add_argument("--extras", default="coupling,td2,df,fp64,fp64e,e2e,cpu",
                   help="comma-separated extras to report after the headline (default all of "
                        "coupling,td2,df,fp64,fp64e,e2e,cpu)")
    p.add_argument("--max-dimers", type=int, default=0,
                   help="keep only the first N dimers of the workload (smaller cases for profiling)")
    p.add_argument("--alias-blocks", action="store_true",
                   help="profiling aid: every dimer reads dimer 0's integral blocks, so the second half runs "
                        "the full dimer grid with a device footprint of one dimer (energies are not the workload's)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            time.sleep(0.2)
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if len(r) > 5 + k and "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        pw = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def gpu_local_cpus(device):
    """The host CPUs the kernel lists as local to this GPU (sysfs), or None."""
    try:
        import torch
        p = torch.cuda.get_device_properties(device)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            text = f.read().strip()
        cpus = set()
        for part in text.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


_FP64_RATE = {}


def fp64_rate(device):
    """The FP64 FMA rate the FP64 form is bound by, measured once per run by
    the library's microbenchmark (mcpt_fp64_fma_rate)."""
    if device not in _FP64_RATE:
        import paper_1409_2700_gb300 as M
        t, ms = M.mcpt_fp64_fma_rate(device)
        _FP64_RATE[device] = {"tflops": t, "kind": f"measured: library DFMA microbenchmark, this run ({ms:.0f} ms)"}
    return _FP64_RATE[device]


# DRAM traffic of the first-half kernel per dimer, from the full ncu capture
# of the current kernel in profiles/k_half_tc_rank_bf16x2_lattice-2x2x2.md
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch over 28 dimers
# of 32 AO / 5 occupied, scaled per dimer).  Only valid for that kernel, form
# and monomer size; the other forms' kernels changed since their captures.
TRAFFIC_PER_DIMER = {("bf16x2", 32, 5): (469.92e6 + 5.563136e6) / 28}


def host_sample(w, dimers):
    """Host inputs for the oracle (host generator)."""
    import synth  # noqa: F401
    items = []
    for d in dimers:
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        A, K = w.blocks(d)
        items.append((A, K, mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc))
    return items


def sample_dimers(w, n):
    step = max(1, w.n_dimers // n)
    return list(range(0, w.n_dimers, step))[:n]


# ------------------------------------------------------------------ reference arm
def reference_arm(args, ws, rank):
    """The FP64 CPU oracle on the machine's host cores, as it stands."""
    if rank != 0:
        return
    import oracle
    import synth
    w = synth.workload(args.workload)
    oracle.build()
    ds = sample_dimers(w, min(args.cpu_sample, 96))   # host generation of the sample stays bounded
    keep, nbytes = [], 0
    for d in ds:                                      # and so does its host memory (4 GB)
        X, Y = w.pairs[d]
        nbytes += 16 * w.nao[X] ** 2 * w.nao[Y] ** 2
        if keep and nbytes > (4 << 30):
            break
        keep.append(d)
    items = host_sample(w, keep)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.dimers_parallel(items[:8])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.dimers_parallel(items)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    v = len(items) * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_dimers": w.n_dimers, "nao": w.nao[0], "nocc": w.nocc[0],
                   "sample_dimers": len(items), "inputs": "host RAM"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{len(items)} evenly spaced dimers of {args.workload} per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def our_arm(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1409_2700_gb300 as M
    import synth
    import synth.device

    torch.cuda.set_device(local)
    w = synth.workload(args.workload)
    if args.max_dimers:
        w.pairs, w.R = w.pairs[:args.max_dimers], w.R[:args.max_dimers]
    # inputs: every dimer's [A | K] blocks resident in HBM (generation untimed)
    if args.alias_blocks:
        buf, offs0 = synth.device.workload_blocks(w, dimers=[0])
        offs = [offs0[0]] * w.n_dimers
    else:
        buf, offs = synth.device.workload_blocks(w)
    torch.cuda.synchronize()
    mons = [w.monomer(X) for X in range(w.n_monomers)]

    stream = torch.cuda.Stream()

    def make_ctx(prec, timing, coupling=False):
        ctx = M.Context(precision=prec, device=local, stream=stream.cuda_stream, validate=False, timing=timing,
                        coupling=coupling, fp64_epilogue=args.fp64_epilogue)
        for m in mons:
            ctx.add_monomer(m.C, m.eps, m.nocc)
        base = buf.data_ptr()
        for d in range(w.n_dimers):
            X, Y = w.pairs[d]
            ctx.add_dimer(X, Y, base + 8 * offs[d], M.MCPT_AO_BLOCKS, on_device=1)
        return ctx

    ctx = make_ctx(args.precision, True)
    for _ in range(args.warmup):
        ctx.run()
    ctx.energies()
    ctx.stats()   # discard warm-up timing

    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                ctx.run()
            e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ws, ms)
    st = ctx.stats()
    mj, mk, pd, tot = ctx.energies()
    clocks = clk.summary()

    ms_step = ms / args.steps
    value = ws * w.n_dimers / (ms_step * 1e-3)
    transform_ms = st.ms[0] / st.runs        # first-half kernel, average per launch (one wave)
    per_launch_bytes = st.alg_bytes / st.waves
    peaks, peak_kind = measured_peaks()
    if args.precision == "fp64":
        # FP64 pipe bound: the measured FP64 FMA rate
        rate = fp64_rate(local)
        achieved = st.alg_flops_half / st.waves / (transform_ms / st.waves * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": rate["tflops"], "unit": "TFLOP/s",
                "frac": achieved / rate["tflops"], "traffic": None, "kernel": "k_half_fp64",
                "peak_kind": rate["kind"]}
    else:
        achieved = per_launch_bytes / (transform_ms / st.waves * 1e-3) / 1e9
        tpd = TRAFFIC_PER_DIMER.get((args.precision, w.nao[0], w.nocc[0]))
        uniform = len(set(w.nao)) == 1 and len(set(w.nocc)) == 1
        traffic = tpd * w.n_dimers / st.waves if (tpd and uniform) else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "k_half_tc_rank" if args.precision in ("tf32", "bf16x3", "bf16x2", "fp64e") else "k_half_fp32c",
                "peak_kind": peak_kind}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "n_dimers": w.n_dimers, "n_monomers": w.n_monomers,
                   "energy_epilogue": "fp64-pipe" if args.fp64_epilogue else "fp32-pairs",
                   "nao": w.nao[0], "nocc": w.nocc[0], "precision": args.precision,
                   "inputs_gb": round(buf.numel() * 8 / 1e9, 2), "l2": "inputs (17.4 GB) larger than L2"},
        "transform_tflops": st.alg_flops / (ms_step * 1e-3) / 1e12,
        "phase_ms_per_step": {"first_half": st.ms[0] / st.runs, "finish": st.ms[1] / st.runs,
                              "reduce": st.ms[2] / st.runs, "run": st.ms[3] / st.runs},
        "roofline": roof,
        "gpu_launches": st.launches,
        "clocks": clocks,
        "lattice_E": {"J": tot[0], "K": tot[1]},
    }

    # ---- accuracy against the stored oracle values (tests/golden)
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        import make_lattice_oracle as golden
        g = None if (args.max_dimers or args.alias_blocks) else golden.load(args.workload)
    except Exception:
        g = None
    if g is not None:
        Eo, to = g
        line["error_eh"] = {"lattice_J": float(tot[0] - to[0]), "lattice_K": float(tot[1] - to[1]),
                            "max_dimer_J": float(np.max(np.abs(pd[:, 0] - Eo[:, 0]))),
                            "max_dimer_K": float(np.max(np.abs(pd[:, 1] - Eo[:, 1]))),
                            "reference": "FP64 oracle, stored per-dimer values"}

    # ---- the same runs replayed as a captured CUDA graph (the library's default
    # when per-phase timing is off); reported beside the eagerly timed value
    gctx = make_ctx(args.precision, False)
    for _ in range(args.warmup):
        gctx.run()
    gctx.energies()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g0.record(stream)
        for _ in range(args.steps):
            gctx.run()
        g1.record(stream)
    torch.cuda.synchronize()
    gms = g0.elapsed_time(g1) / args.steps
    line["graph"] = {"value": w.n_dimers / (gms * 1e-3), "unit": UNIT, "ms_per_step": gms}
    gctx.close()

    extras = set() if args.no_extras else set(x for x in args.extras.split(",") if x)
    if rank == 0 and "coupling" in extras:
        # ---- the dimer -> monomer doubles coupling of Eq. (tm2) at first order on
        # the same inputs: the same runs with coupling on, the difference timed
        cc = make_ctx(args.precision, False, coupling=True)
        cc.run()
        cmj = cc.energies()[0]
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            c0.record(stream)
            for _ in range(args.steps):
                cc.run()
            c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / args.steps
        cflops = 0.0
        for X, Y in w.pairs:
            mX = w.nocc[X] * (w.nao[X] - w.nocc[X])
            mY = w.nocc[Y] * (w.nao[Y] - w.nocc[Y])
            cflops += 2 * 2 * (mX * mX * mY + mY * mY * mX)
        trace_err = max(abs(np.trace(cc.coupling(X, w.nao[X], w.nocc[X])) - cmj[X]) / abs(cmj[X])
                        for X in range(w.n_monomers))
        line["coupling"] = {"ms_per_step": cms, "extra_ms_per_step": cms - gms,
                            "tflops": cflops / ((cms - gms) * 1e-3) / 1e12 if cms > gms else None,
                            "alg_gflop_per_step": cflops / 1e9,
                            "max_rel_trace_minus_monomer_EJ": trace_err,
                            "what": "R_X = sum_Y (T V^t + V T^t) of Eq. (tm2) at T = vD, every monomer"}
        # ---- the singles environment term of Eq. (tm1) from the same stored
        # (ia|kc), for seeded amplitudes: host-synchronous calls (amplitudes in,
        # result out) timed by wall clock; s(2t) = 2 s(t) holds bit for bit
        trng = np.random.default_rng(7)
        t1 = [trng.standard_normal((w.nocc[X], w.nao[X] - w.nocc[X])) * 0.01 for X in range(w.n_monomers)]
        s1 = cc.singles(t1)
        reps = 10
        t0 = time.perf_counter()
        for _ in range(reps):
            cc.singles(t1)
        sms = (time.perf_counter() - t0) / reps * 1e3
        s2 = cc.singles([2.0 * x for x in t1])
        vbytes = sum(2 * 4 * (w.nocc[X] * (w.nao[X] - w.nocc[X])) * (w.nocc[Y] * (w.nao[Y] - w.nocc[Y]))
                     for X, Y in w.pairs) * (2 if args.precision == "fp64" else 1)
        line["coupling"]["singles"] = {
            "ms_per_call": sms, "alg_bytes_per_call": vbytes,
            "linear_bitwise": bool(all(np.array_equal(b, 2.0 * a) for a, b in zip(s1, s2))),
            "what": "s_X = sum_Y sum_kc (ia|kc) t_kc(Y) of Eq. (tm1), every monomer; wall clock per "
                    "mcpt_singles call including the amplitude and result copies"}
        cc.close()

    # ---- the dimer doubles iteration of Eq. (td2) on the same inputs, with
    # synthetic monomer matrices: 10 Jacobi steps in this form's arithmetic
    # and in FP64; two sampled dimers against the oracle
    if rank == 0 and "td2" in extras:
        import oracle
        oracle.build()
        md = {X: synth.monomer_doubles(X, w.nao[X], w.nocc[X]) for X in range(w.n_monomers)}
        nit = 10
        td = {}
        samp = [0, w.n_dimers - 1]
        refs = []
        for d in samp:
            X, Y = w.pairs[d]
            n4 = 2 * w.nao[X] ** 2 * w.nao[Y] ** 2
            blk = buf[offs[d]:offs[d] + n4].cpu().numpy()
            A = blk[:n4 // 2].reshape(w.nao[X], w.nao[X], w.nao[Y], w.nao[Y])
            K = blk[n4 // 2:].reshape(w.nao[X], w.nao[Y], w.nao[Y], w.nao[X])
            refs.append(oracle.td2(A, K, mons[X].C, mons[X].eps, mons[Y].C, mons[Y].eps, mons[X].nocc,
                                   mons[Y].nocc, nit, md[X][0], md[Y][0], md[X][1], md[Y][1])[1])
        flops = 0.0
        for X, Y in w.pairs:
            nX, nY, oX, oY = w.nao[X], w.nao[Y], w.nocc[X], w.nocc[Y]
            vX, vY = nX - oX, nY - oY
            mX, mY = oX * vX, oY * vY
            flops += 2 * (2 * nX ** 2 * nY ** 3 + 2 * nX ** 3 * nY ** 2)          # MO transformation of A
            flops += 2 * (nX * nY * nY * vX * nX + vX * nX * nY * oY * nY + oY * vX * nX * vY * nY
                          + vY * oY * vX * oX * nX)                               # (ib|ja) from K
            flops += 2 * mX * mY * (mX + mY)                                      # monomer-amplitude source
            flops += nit * 2 * (vX * vY * oX * oY * vX * vY + oX * oY * vX * vY * oX * oY
                                + mX * mY * (oX * vY + vX * oY) + mX * mY * (mX + mY))  # ladders, mixed, ring
        for prec in ([args.precision, "fp64"] if args.precision != "fp64" else ["fp64"]):
            tctx = make_ctx(prec, False)
            for X in range(w.n_monomers):
                tctx.set_monomer_doubles(X, *md[X])
            tctx.td2(1)                          # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            got, dl = tctx.td2(nit)
            dt = time.perf_counter() - t0
            tctx.close()
            err = max(abs(got[d, 0] - r[0]) / abs(r[0]) for d, r in zip(samp, refs))
            td[prec] = {"s_per_call": dt, "dimers_per_s": w.n_dimers / dt, "tflops": flops / dt / 1e12,
                        "final_step_max_dT": float(dl[-1]), "sample_max_rel_err_EJ": float(err)}
        line["td2"] = {"iterations": nit, "alg_gflop": flops / 1e9, "forms": td,
                       "what": "Eq. (td2) dimer doubles amplitudes by Jacobi steps from zero for every dimer "
                               "(full MO transformation of the Coulomb block, ladders, mixed Coulomb terms, "
                               "synthetic monomer ring and amplitude matrices), energies at the final "
                               "amplitudes; wall clock per mcpt_td2 call; the error is against the FP64 oracle "
                               "on the first and last dimer"}

    # ---- the density-fitted route on the same lattice: every dimer's
    # three-index factors resident on the device (generated, untimed), the
    # terms from them; checked against the stored four-index oracle values
    if rank == 0 and "df" in extras:
        import synth.device as sdev
        Bs = []
        for d in range(w.n_dimers):
            X, Y = w.pairs[d]
            Bs.append(sdev.factors(X, Y, w.nao[X], w.nao[Y], seed=w.seed))
        torch.cuda.synchronize()
        df = {}
        dbytes = sum(B.numel() * 8 for B in Bs)
        for prec in ([args.precision, "fp64"] if args.precision != "fp64" else ["fp64"]):
            dctx = M.Context(precision=prec, device=local, stream=stream.cuda_stream, validate=False, fp64_epilogue=args.fp64_epilogue)
            for m in mons:
                dctx.add_monomer(m.C, m.eps, m.nocc)
            for d in range(w.n_dimers):
                X, Y = w.pairs[d]
                dctx.add_dimer_df(X, Y, Bs[d].data_ptr(), Bs[d].shape[0], synth.scale_for_distance(w.R[d]),
                                  on_device=1)
            for _ in range(args.warmup):
                dctx.run_df()
            reps = 5
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                dctx.run_df()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            _, _, dpd, dtot = dctx.df_energies()
            dctx.close()
            ent = {"value": w.n_dimers / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                   "achieved_gbs": dbytes / (ms * 1e-3) / 1e9, "bytes_per_step": dbytes}
            if g is not None:
                ent["max_rel_err_vs_four_index_oracle"] = float(np.max(np.abs(dpd - g[0]) / np.abs(g[0][:, :1])))
                ent["lattice_J_err_eh"] = float(dtot[0] - g[1][0])
            df[prec] = ent
        del Bs
        line["df"] = {"forms": df, "what": "density-fitted route (three-index factors B^Q, naux 192, 6.3 MB per "
                                           "dimer, device-resident): half-transformations, pair contractions over "
                                           "Q with the FP64 energy epilogue, per-monomer reduction; mcpt_run_df "
                                           "timed with CUDA events (it waits for its work)"}

    # ---- the plain FP64 GPU form on the same resident inputs
    if rank == 0 and "fp64" in extras and args.precision != "fp64":
        c64 = make_ctx("fp64", True)
        c64.run()
        c64.energies()
        c64.stats()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n64 = max(2, args.steps // 4)
        with torch.cuda.stream(stream):
            f0.record(stream)
            for _ in range(n64):
                c64.run()
            f1.record(stream)
        torch.cuda.synchronize()
        s64 = c64.stats()
        _, _, pd64, tot64 = c64.energies()
        ms64 = f0.elapsed_time(f1) / n64
        fp64 = {"value": w.n_dimers / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "transform_tflops": s64.alg_flops / (ms64 * 1e-3) / 1e12,
                "first_half_ms": s64.ms[0] / s64.runs}
        rate = fp64_rate(local)
        a64 = s64.alg_flops_half / (s64.ms[0] / s64.runs * 1e-3) / 1e12
        fp64["roofline"] = {"bound": "alu", "achieved": a64, "peak": rate["tflops"], "unit": "TFLOP/s",
                            "frac": a64 / rate["tflops"], "kernel": "k_half_fp64", "peak_kind": rate["kind"]}
        if g is not None:
            fp64["error_eh_lattice_J"] = float(tot64[0] - g[1][0])
        line["fp64_form"] = fp64
        c64.close()

    if rank == 0 and "e2e" in extras:
        # ---- end to end through the C ABI from pinned host buffers, in two
        # input layouts: the blocks (BLOCKS) and their unique elements under
        # the real-orbital pair symmetry (PACKED, expanded on the device)
        host = torch.empty(buf.numel(), dtype=torch.float64, pin_memory=True)
        host.copy_(buf)
        shapes = {}
        poffs, ptot = [], 0
        for d in range(w.n_dimers):
            X, Y = w.pairs[d]
            key = (w.nao[X], w.nao[Y])
            if key not in shapes:
                shapes[key] = torch.from_numpy(synth.packed_gather_index(*key)).to(buf.device)
            poffs.append(ptot)
            ptot += shapes[key].numel()
        phost = torch.empty(ptot, dtype=torch.float64, pin_memory=True)
        for d in range(w.n_dimers):                 # input preparation (untimed): gather the unique elements
            X, Y = w.pairs[d]
            idx = shapes[(w.nao[X], w.nao[Y])]
            phost[poffs[d]:poffs[d] + idx.numel()].copy_(buf[offs[d]:offs[d] + 2 * w.nao[X] ** 2 * w.nao[Y] ** 2][idx])
        torch.cuda.synchronize()
        d2h = 8 * (2 * w.n_monomers + 2 * w.n_dimers + 2)
        del ctx
        torch.cuda.synchronize()

        def e2e(layout, base, doffs):
            # one context for the whole sequence (set up untimed: monomers,
            # dimers, the plan and its graph); every timed step copies that
            # step's integrals from pinned host memory into it
            # (mcpt_update_dimer, asynchronous), runs, and reads the energies back
            c = M.Context(precision=args.precision, device=local, validate=False, fp64_epilogue=args.fp64_epilogue)
            for m in mons:
                c.add_monomer(m.C, m.eps, m.nocc)
            for d in range(w.n_dimers):
                X, Y = w.pairs[d]
                c.add_dimer(X, Y, base + 8 * doffs[d], layout, on_device=0)
            c.run()
            c.energies()
            ts, same = [], True
            for k in range(args.e2e_steps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c.update_dimers(0, w.n_dimers, base, doffs, layout, asynchronous=True)
                c.run()
                out = c.energies()
                t1 = time.perf_counter()
                same = same and bool(np.array_equal(out[2], pd))
                if k > 0:
                    ts.append(t1 - t0)
            c.close()
            return statistics.median(ts), len(ts), same

        blk_bytes = sum(2 * 8 * (w.nao[w.pairs[d][0]] ** 2) * (w.nao[w.pairs[d][1]] ** 2) for d in range(w.n_dimers))
        ps, pn, psame = e2e(M.MCPT_AO_PACKED, phost.data_ptr(), poffs)
        bs, bn, bsame = e2e(M.MCPT_AO_BLOCKS, host.data_ptr(), offs)
        line["e2e"] = {"value": w.n_dimers / ps, "unit": UNIT, "h2d_bytes_per_step": 8 * ptot,
                       "d2h_bytes_per_step": d2h, "s_per_step": ps, "steps": pn,
                       "terms_equal_resident_run": psame,
                       "per_step": "mcpt_update_dimers of every dimer's symmetry-packed integrals (MCPT_AO_PACKED: "
                                   "the unique elements, back to back, copied in 256 MB chunks and expanded on the "
                                   "device) from pinned host memory (asynchronous), mcpt_run, mcpt_energies; context, "
                                   "monomers and plan set up once"}
        line["e2e_blocks"] = {"value": w.n_dimers / bs, "unit": UNIT, "h2d_bytes_per_step": blk_bytes,
                              "d2h_bytes_per_step": d2h, "s_per_step": bs, "steps": bn,
                              "terms_equal_resident_run": bsame,
                              "per_step": "the same with the BLOCKS layout (both blocks in full)"}
        del host, phost

    if rank == 0 and "cpu" in extras:
        # ---- the oracle on the host cores, bounded sample
        import oracle
        oracle.build()
        ds = sample_dimers(w, args.cpu_sample)
        n4 = 32 ** 4
        Eo = np.empty((len(ds), 2))
        tc = 0.0
        for c0 in range(0, len(ds), 64):          # bounded host memory: 64 dimers at a time
            items = []
            for d in ds[c0:c0 + 64]:
                X, Y = w.pairs[d]
                mX, mY = mons[X], mons[Y]
                blk = buf[offs[d]:offs[d] + 2 * n4].cpu().numpy()
                items.append((blk[:n4].reshape(32, 32, 32, 32), blk[n4:].reshape(32, 32, 32, 32),
                              mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc))
            t0 = time.perf_counter()
            Eo[c0:c0 + len(items)] = oracle.dimers_parallel(items)
            tc += time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(ds) / tc, "unit": UNIT, "cores": oracle.max_threads(),
                                "kind": "oracle",
                                "sample": f"{len(ds)} evenly spaced dimers of {args.workload}, one pass "
                                          f"({tc:.1f} s wall)"}
        line["sample_error_eh"] = {"max_dimer_J": float(np.max(np.abs(pd[ds, 0] - Eo[:, 0]))),
                                   "max_dimer_K": float(np.max(np.abs(pd[ds, 1] - Eo[:, 1])))}
    if rank == 0:
        print(json.dumps(line))


# ------------------------------------------------------------------ streamed workloads
# Workloads whose integral blocks exceed device memory (706 GB for the
# 10x10x10 lattice) run in waves through one context: every dimer is
# registered once with an address inside one wave buffer, and a producer
# writes each wave's blocks there (device generation, untimed) before the
# wave runs.  A step is one wave: one pass of the whole path over one batch
# of the workload's dimers (about WAVE_BUDGET bytes of integrals).  Steps
# walk the waves in order and wrap around; when the steps end before the
# lattice does, the remaining waves run untimed so that the lattice energy
# can be checked against the stored oracle values.
STREAMED = {"lattice-10x10x10-cheb2", "uneven-4096", "lattice-7x7x7-cheb1-ao128"}
WAVE_BUDGET = 36 << 30


def _alg_bytes(w, d0, n):
    return float(sum(2 * 8 * w.nao[w.pairs[d][0]] ** 2 * w.nao[w.pairs[d][1]] ** 2 for d in range(d0, d0 + n)))


def _tune_lines(path):
    if not path or not os.path.exists(path):
        return None
    with open(path) as f:
        return [ln.strip() for ln in f if ln.strip()]


def _alg_flops(w, d0, n):
    """(all, first half) algorithmic transform flops of dimers d0 .. d0+n-1:
    the occupied-first factorised count, both forms."""
    tot = half = 0.0
    for d in range(d0, d0 + n):
        X, Y = w.pairs[d]
        nx, ny, ox, oy = w.nao[X], w.nao[Y], w.nocc[X], w.nocc[Y]
        vx, vy = nx - ox, ny - oy
        h = 4.0 * (nx * nx * ny * ny * oy + ox * nx * nx * ny * oy)
        half += h
        tot += h + 4.0 * (ox * nx * oy * ny * vy + ox * vx * oy * vy * nx)
    return tot, half


def streamed_arm(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1409_2700_gb300 as M
    import synth
    import synth.device
    from paper_1409_2700_gb300.stream import Streamed

    from paper_1409_2700_gb300.stream import block_elems, plan_waves
    torch.cuda.set_device(local)
    w = synth.workload(args.workload)
    if args.max_dimers:
        w.pairs, w.R = w.pairs[:args.max_dimers], w.R[:args.max_dimers]
    n_all = w.n_dimers
    # a lattice whose generation alone would take many minutes per pass (the
    # 128-AO one: 4.3 GB and ~0.2 s of FP64 GEMMs per dimer) runs the dimers
    # of the waves the steps cover, not the whole list
    budget = int(args.wave_gb * (1 << 30))
    full_waves = plan_waves([block_elems(w.nao[X], w.nao[Y]) for X, Y in w.pairs], budget // 8)[0]
    subset = len(full_waves) > args.max_waves
    if subset:
        keep = sum(c for _, c in full_waves[:max(1, args.steps)])
        w.pairs, w.R = w.pairs[:keep], w.R[:keep]
    extras = set() if args.no_extras else set(x for x in args.extras.split(",") if x)
    if any(n > 96 for n in w.nao):
        extras.discard("fp64")                      # the FP64 form handles monomers of up to 96 AO
    stream = torch.cuda.Stream()
    mons = [w.monomer(X) for X in range(w.n_monomers)]

    tune = os.path.join(tempfile.gettempdir(), f"mcpt_tune_{os.getpid()}.txt") if args.tune else None

    def make_ctx(prec, timing, graphs=True):
        c = M.Context(precision=prec, device=local, stream=stream.cuda_stream, validate=False, timing=timing,
                      graphs=graphs, tune_cache=tune if prec != "fp64" else None, fp64_epilogue=args.fp64_epilogue)
        for m in mons:
            c.add_monomer(m.C, m.eps, m.nocc)
        return c

    # the timed value: each wave's run replayed as its plan's CUDA graph; a
    # second context with per-phase CUDA events (same launch choices) runs the
    # same waves for the phase times and the roofline
    ctx = make_ctx(args.precision, False)
    ctx_t = make_ctx(args.precision, True)
    ctxs = [ctx, ctx_t]
    c64 = None
    if rank == 0 and "fp64" in extras and args.precision != "fp64":
        c64 = make_ctx("fp64", True)
        ctxs.append(c64)
    # the FP64-emulating tensor-core form (monomers of up to 64 AO, 5 occupied) on the same waves
    cE = None
    if (rank == 0 and "fp64e" in extras and args.precision != "fp64e" and max(w.nao) <= 64 and max(w.nocc) <= 5):
        cE = make_ctx("fp64e", True)
        ctxs.append(cE)
    with torch.cuda.stream(stream):
        st = Streamed(ctxs, w.pairs, w.nao, budget)
        nw = len(st)
        st.buf.zero_()
        synth.device.fill_views(w, st.views(0))
        # plans of every wave built before timing (runs on whatever the buffer holds)
        for k in range(nw):
            st.run(k)
        for _ in range(max(args.warmup, 3)):
            ctx.run(*st.waves[0])
            ctx_t.run(*st.waves[0])
        stream.synchronize()
        for c in ctxs[1:]:
            c.stats()
        ev, ev64, done, done64, evE, doneE = [], [], set(), set(), [], set()
        t_gen, timed_dimers, timed_bytes, timed_flops, timed_half, filled = 0.0, 0, 0.0, 0.0, 0.0, 0
        wave_flops = [_alg_flops(w, *st.waves[k]) for k in range(nw)]
        with Clocks(local) as clk:
            for step in range(args.steps):
                k = step % nw
                if filled != k:                            # the buffer holds wave `filled`
                    t0 = time.perf_counter()
                    synth.device.fill_views(w, st.views(k))
                    stream.synchronize()
                    t_gen += time.perf_counter() - t0
                    filled = k
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.run(*st.waves[k])
                e1.record(stream)
                ev.append((e0, e1))
                ctx_t.run(*st.waves[k])
                timed_dimers += st.waves[k][1]
                timed_bytes += _alg_bytes(w, *st.waves[k])
                timed_flops += wave_flops[k][0]
                timed_half += wave_flops[k][1]
                done.add(k)
                if c64 is not None and k not in done64:
                    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    f0.record(stream)
                    c64.run(*st.waves[k])
                    f1.record(stream)
                    ev64.append((f0, f1, st.waves[k][1]))
                    done64.add(k)
                if cE is not None and k not in doneE:
                    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    f0.record(stream)
                    cE.run(*st.waves[k])
                    f1.record(stream)
                    evE.append((f0, f1, st.waves[k][1], k))
                    doneE.add(k)
            stream.synchronize()
        clocks = clk.summary()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        stt = ctx_t.stats()
        s64 = c64.stats() if c64 is not None else None
        sE = cE.stats() if cE is not None else None
        # the waves the steps did not reach, untimed, so that the lattice is complete
        for k in range(nw):
            if k in done and (c64 is None or k in done64) and (cE is None or k in doneE):
                continue
            if filled != k:
                synth.device.fill_views(w, st.views(k))
                filled = k
            if k not in done:
                ctx.run(*st.waves[k])
                ctx_t.run(*st.waves[k])
            if c64 is not None and k not in done64:
                c64.run(*st.waves[k])
            if cE is not None and k not in doneE:
                cE.run(*st.waves[k])
        stream.synchronize()

    mj, mk, pd, tot = ctx.energies()
    nsteps = len(ev)
    ms = max_over_ranks(ws, ms)
    ms_step = ms / nsteps
    peaks, peak_kind = measured_peaks()
    first_half_ms = stt.ms[0]
    if args.precision == "fp64":
        rate = fp64_rate(local)
        achieved = timed_half / (first_half_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": rate["tflops"], "unit": "TFLOP/s",
                "frac": achieved / rate["tflops"], "traffic": None, "kernel": "k_half_fp64",
                "peak_kind": rate["kind"]}
    else:
        achieved = timed_bytes / (first_half_ms * 1e-3) / 1e9
        tpd = TRAFFIC_PER_DIMER.get((args.precision, w.nao[0], w.nocc[0]))
        uniform = len(set(w.nao)) == 1 and len(set(w.nocc)) == 1
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": tpd * timed_dimers / nsteps if (tpd and uniform) else None,
                "kernel": "k_half_tc_rank" if args.precision in ("tf32", "bf16x3", "bf16x2", "fp64e") else "k_half_fp32c",
                "peak_kind": peak_kind,
                "per": "one wave's first-half launch (traffic scaled from the ncu capture per dimer)"}
    line = {
        "metric": METRIC, "value": ws * timed_dimers / (ms * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": nsteps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "n_dimers": w.n_dimers, "n_monomers": w.n_monomers,
                   "energy_epilogue": "fp64-pipe" if args.fp64_epilogue else "fp32-pairs",
                   "nao": sorted(set(w.nao)), "nocc": sorted(set(w.nocc)), "precision": args.precision,
                   "inputs_gb": round(_alg_bytes(w, 0, w.n_dimers) / 1e9, 1), "waves": nw,
                   "dimers_per_step": round(timed_dimers / nsteps, 1),
                   "dimers_run": w.n_dimers if not subset else
                   f"the first {w.n_dimers} of {n_all} (the waves the steps cover; {len(full_waves)} waves in all)",
                   "step": "one wave: every dimer of the wave through the whole path (first half, second half "
                           "with FP64 denominators and energies, per-monomer reduction); waves in lattice order",
                   "timed": "CUDA events around each wave's run; on-device generation of each wave untimed",
                   "l2": "inputs (tens of GB per wave) larger than L2"},
        "phase_ms_per_step": {"first_half": stt.ms[0] / nsteps, "finish": stt.ms[1] / nsteps,
                              "reduce": stt.ms[2] / nsteps, "run": stt.ms[3] / nsteps,
                              "note": "eagerly launched twin context with per-phase CUDA events"},
        "graphs": "each wave's run replayed as its plan's captured CUDA graph",
        "autotuner": _tune_lines(tune),
        "transform_tflops": timed_flops / (ms * 1e-3) / 1e12,
        "generation_s_per_step": t_gen / nsteps,
        "roofline": roof,
        "gpu_launches": stt.launches,   # the twin's count: a graph replays the same launches
        "clocks": clocks,
        "lattice_E": {"J": tot[0], "K": tot[1]},
    }

    # ---- accuracy against the stored oracle values (tests/golden), every dimer
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        import make_lattice_oracle as golden
        g = None if args.max_dimers else golden.load(args.workload)
    except Exception:
        g = None
    if g is not None:
        Eo, to = g
        nd = min(len(Eo), w.n_dimers)
        err = {"max_dimer_J": float(np.max(np.abs(pd[:nd, 0] - Eo[:nd, 0]))),
               "max_dimer_K": float(np.max(np.abs(pd[:nd, 1] - Eo[:nd, 1]))),
               "max_dimer_rel_J": float(np.max(np.abs(pd[:nd, 0] - Eo[:nd, 0]) / np.abs(Eo[:nd, 0]))),
               "sum_J_of_those_dimers": float(pd[:nd, 0].sum() - Eo[:nd, 0].sum())}
        if not subset and nd == w.n_dimers and to[0] is not None:
            err["lattice_J"] = float(tot[0] - to[0])
            err["lattice_K"] = float(tot[1] - to[1])
        err["reference"] = f"FP64 oracle (factor route), stored values of {nd} of the {w.n_dimers} dimers run"
        line["error_eh"] = err

    # ---- the plain FP64 GPU form on the same waves (each wave once)
    if c64 is not None:
        _, _, pd64, tot64 = c64.energies()
        ms64 = sum(a.elapsed_time(b) for a, b, _ in ev64)
        n64 = sum(n for _, _, n in ev64)
        rate = fp64_rate(local)
        half64 = sum(wave_flops[k][1] for k in done64)
        fp64 = {"value": n64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / len(ev64), "waves": len(ev64),
                "first_half_ms_per_step": s64.ms[0] / len(ev64),
                "roofline": {"bound": "alu", "achieved": half64 / (s64.ms[0] * 1e-3) / 1e12, "peak": rate["tflops"],
                             "unit": "TFLOP/s", "kernel": "k_half_fp64", "peak_kind": rate["kind"]}}
        fp64["roofline"]["frac"] = fp64["roofline"]["achieved"] / rate["tflops"]
        if g is not None:
            nd = min(len(g[0]), w.n_dimers)
            if not subset and nd == w.n_dimers and g[1][0] is not None:
                fp64["error_eh_lattice_J"] = float(tot64[0] - g[1][0])
            fp64["max_dimer_rel_J"] = float(np.max(np.abs(pd64[:nd, 0] - g[0][:nd, 0]) / np.abs(g[0][:nd, 0])))
        line["fp64_form"] = fp64

    # ---- the FP64-emulating tensor-core form on the same waves (each wave once)
    if cE is not None:
        _, _, pdE, totE = cE.energies()
        msE = sum(a.elapsed_time(b) for a, b, _, _ in evE)
        nE = sum(n for _, _, n, _ in evE)
        bytesE = sum(_alg_bytes(w, *st.waves[k]) for _, _, _, k in evE)
        fE = {"value": nE / (msE * 1e-3), "unit": UNIT, "ms_per_step": msE / len(evE), "waves": len(evE),
              "first_half_ms_per_step": sE.ms[0] / len(evE), "finish_ms_per_step": sE.ms[1] / len(evE),
              "roofline": {"bound": "hbm", "achieved": bytesE / (sE.ms[0] * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "kernel": "k_half_tc_rank (FP64E)", "peak_kind": peak_kind},
              "what": "FP64-accurate form on the tensor cores: 48-bit fixed-point byte digits, exact tcgen05 "
                      "FP16 sums, FP32-pair epilogue and second half, FP64 sums"}
        fE["roofline"]["frac"] = fE["roofline"]["achieved"] / peaks["hbm_gbs"]
        if c64 is not None:
            fE["speedup_vs_fp64_form"] = fE["value"] / line["fp64_form"]["value"]
        if g is not None:
            nd = min(len(g[0]), w.n_dimers)
            if not subset and nd == w.n_dimers and g[1][0] is not None:
                fE["error_eh_lattice_J"] = float(totE[0] - g[1][0])
                fE["error_eh_lattice_K"] = float(totE[1] - g[1][1])
            fE["max_dimer_rel_J"] = float(np.max(np.abs(pdE[:nd, 0] - g[0][:nd, 0]) / np.abs(g[0][:nd, 0])))
        line["fp64e_form"] = fE

    # ---- the oracle on the host cores, part 1: evenly spaced dimers of the
    # wave in the buffer, their four-index blocks copied to the host (the
    # oracle runs after the end-to-end leg, so that its threads and buffers
    # do not sit between that leg and the device)
    cpu_items = None
    if rank == 0 and "cpu" in extras:
        first, count = st.waves[filled]
        ds = [first + k for k in range(0, count, max(1, count // max(1, args.cpu_sample)))][:args.cpu_sample]
        cpu_items = []
        for d in ds:
            X, Y = w.pairs[d]
            nX, nY = w.nao[X], w.nao[Y]
            blk = st.buf[st.offs[d]:st.offs[d] + 2 * nX * nX * nY * nY].cpu().numpy()
            cpu_items.append((d, (blk[:nX * nX * nY * nY].reshape(nX, nX, nY, nY),
                                  blk[nX * nX * nY * nY:].reshape(nX, nY, nY, nX),
                                  mons[X].C, mons[X].eps, mons[Y].C, mons[Y].eps, mons[X].nocc, mons[Y].nocc)))

    # ---- end to end through the C ABI from pinned host buffers: a context
    # holding the dimers of the first waves, each step one wave: every dimer's
    # symmetry-packed integrals copied from pinned host memory
    # (mcpt_update_dimer, asynchronous, expanded on the device), mcpt_run of
    # the wave, mcpt_energies read back
    if rank == 0 and "e2e" in extras:
        affinity = os.sched_getaffinity(0)
        local_cpus = gpu_local_cpus(local)
        if local_cpus:
            os.sched_setaffinity(0, local_cpus)     # pinned buffers on the GPU's own host node
        ne = max(1, min(args.e2e_steps, nw, 2))
        idx = {}
        hosts, poffs = [], []
        for k in range(ne):
            if filled != k:
                synth.device.fill_views(w, st.views(k))
                filled = k
            first, count = st.waves[k]
            offs_k, tot_k = [], 0
            for d in range(first, first + count):
                key = (w.nao[w.pairs[d][0]], w.nao[w.pairs[d][1]])
                if key not in idx:
                    idx[key] = torch.from_numpy(synth.packed_gather_index(*key)).to(st.buf.device)
                offs_k.append(tot_k)
                tot_k += idx[key].numel()
            hk = torch.empty(tot_k, dtype=torch.float64, pin_memory=True)
            for j, d in enumerate(range(first, first + count)):      # input preparation (untimed)
                key = (w.nao[w.pairs[d][0]], w.nao[w.pairs[d][1]])
                hk[offs_k[j]:offs_k[j] + idx[key].numel()].copy_(st.buf[st.offs[d]:st.offs[d] + st.elems[d]][idx[key]])
            stream.synchronize()
            hosts.append(hk)
            poffs.append(offs_k)
        del idx
        wl = list(st.waves)
        for c in ctxs:
            c.close()
        del st
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        ce = M.Context(precision=args.precision, device=local, validate=False, fp64_epilogue=args.fp64_epilogue)
        for m in mons:
            ce.add_monomer(m.C, m.eps, m.nocc)
        ranges, base_id = [], 0
        wave_of = []
        for k in range(ne):
            first, count = wl[k]
            for j, d in enumerate(range(first, first + count)):
                X, Y = w.pairs[d]
                ce.add_dimer(X, Y, hosts[k].data_ptr() + 8 * poffs[k][j], M.MCPT_AO_PACKED, on_device=0)
            ranges.append((base_id, count, first))
            base_id += count
        for lo, n, _ in ranges:
            ce.run(lo, n)
        ce.energies()
        ts, same, h2d = [], True, 0
        for rep in range(2):
            for k, (lo, n, first) in enumerate(ranges):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ce.update_dimers(lo, n, hosts[k].data_ptr(), poffs[k], M.MCPT_AO_PACKED, asynchronous=True)
                ce.run(lo, n)
                out = ce.energies()
                t1 = time.perf_counter()
                same = same and bool(np.array_equal(out[2][lo:lo + n], pd[first:first + n]))
                if rep > 0 or ne == 1:
                    ts.append((t1 - t0, n, hosts[k].numel() * 8))
        ce.close()
        e2e_s = sum(t for t, _, _ in ts)
        line["e2e"] = {"value": sum(n for _, n, _ in ts) / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": sum(b for _, _, b in ts) / len(ts),
                       "d2h_bytes_per_step": 8 * (2 * w.n_monomers + 2 * base_id + 2),
                       "s_per_step": e2e_s / len(ts), "steps": len(ts),
                       "terms_equal_streamed_run": same,
                       "per_step": "one wave: mcpt_update_dimers of its dimers from pinned host memory "
                                   "(MCPT_AO_PACKED: the unique elements, back to back, copied in 256 MB chunks and "
                                   "expanded on the device, asynchronous), mcpt_run of the wave, mcpt_energies",
                       "host_threads": "the GPU's local CPUs" if local_cpus else "unrestricted"}
        del hosts
        os.sched_setaffinity(0, affinity)
    else:
        for c in ctxs:
            c.close()
        del st
    # ---- the oracle on the host cores, part 2: about 10 s of CPU work
    if cpu_items:
        import oracle
        oracle.build()
        Eo_s, done_s, tc = [], [], 0.0
        for c0 in range(0, len(cpu_items), 64):
            chunk = cpu_items[c0:c0 + 64]
            t0 = time.perf_counter()
            Eo_s.append(oracle.dimers_parallel([it for _, it in chunk]))
            tc += time.perf_counter() - t0
            done_s += [d for d, _ in chunk]
            if tc > 12.0:
                break
        del cpu_items
        Eo_s = np.concatenate(Eo_s)
        line["cpu_baseline"] = {"value": len(done_s) / tc, "unit": UNIT, "cores": oracle.max_threads(),
                                "kind": "oracle",
                                "sample": f"{len(done_s)} evenly spaced dimers of one wave of {args.workload} "
                                          f"(four-index FP64 oracle from the device blocks, {tc:.1f} s wall)"}
        line["sample_error_eh"] = {"max_dimer_J": float(np.max(np.abs(pd[done_s, 0] - Eo_s[:, 0]))),
                                   "max_dimer_K": float(np.max(np.abs(pd[done_s, 1] - Eo_s[:, 1]))),
                                   "dimers": len(done_s), "reference": "four-index FP64 oracle"}
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
    elif args.workload in STREAMED:
        streamed_arm(args, ws, rank, local)
    else:
        our_arm(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
