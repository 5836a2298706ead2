#!/usr/bin/env python
"""Throughput of the streaming cyclic-correlation estimator on one GB300 (or N, one per rank).

Workload (one step): a GMSK stream of 2^26 complex64 samples (BT 0.3, 8 samples/symbol,
carrier offset 0.05, 10 dB) pushed in 2^16-sample chunks through cyc_push, lags 0..127,
1024 cycle frequencies -0.5 + k/1024, both forms, FP64 running sums, then cyc_read.
The input (512 MB) is resident in HBM and larger than L2.

Metric: algorithmic complex MACs per second (one CMAC = one (a, m, n) term per form,
counted over distinct a mod 1), in GMAC/s; also samples/s.  The tuned projection is
timed beside the plain FP32 path, each with its error against the FP64 oracle on
sampled entries, relative to R^0(0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|fp16|fp32]
  python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cyclic-corr GMAC/s and Msamples/s, tuned vs plain FP32 at <=1e-4 err; p99 lat"
UNIT = "GMAC/s"
T_SAMPLES = 1 << 26
CHUNK = 1 << 16
PASS = 1 << 20                         # the stream's max_chunk: 16 pushes projected per launch
NLAGS, NALPHAS, NFORMS = 128, 1024, 2
FLOPS_PER_CMAC = 8                     # one complex multiply-add (the algorithmic unit)
TC_PASSES = {"bf16x3": 3, "fp16": 1}   # tensor-core products per real product
# The tensor-core projection takes a and -a together: a pair costs 2 real multiply-adds per
# complex term and pass (4 flop) instead of the 4 (8 flop) of a complex product; on the
# benchmark grid -1/2 + k/1024 every cycle frequency is in a pair (or the real unit {0, 1/2}).
TC_EXEC_FLOPS_PER_CMAC_PASS = 4
TOL = {"fp32": 1e-5, "bf16x3": 1e-4, "fp16": 1e-2}

# dram__bytes_read.sum + dram__bytes_write.sum per projection launch from one ncu capture,
# valid only for the kernel source it was taken on (sha256 prefix of the .cu file) and the
# samples one launch projects.
TRAFFIC = {
    "proj_tc@1c7ae1991702@1048576": 8481536 + 3235584,   # profiles/proj_tc_bf16x3_cfg1_ncu.md
}


def workload_config(precision):
    return {
        "workload": "cfg1 GMSK stream: %d complex64 samples pushed in 2^16-sample chunks, "
                    "lags 0..127, 1024 cycle freqs -0.5+k/1024, CONV+CONJ, FP64 running sums" % ARGS_SAMPLES[0],
        "samples_per_step": ARGS_SAMPLES[0], "chunk": CHUNK, "pass": PASS, "lags": NLAGS, "cycle_freqs": NALPHAS,
        "forms": NFORMS, "projection": precision,
        "l2": "inputs larger than L2 (%d MB stream per step, 129 MB L2)" % (ARGS_SAMPLES[0] * 8 >> 20)
              if ARGS_SAMPLES[0] * 8 > (129 << 20) else
              "stream of %d MB per step, smaller than L2 (a profiling size)" % (ARGS_SAMPLES[0] * 8 >> 20),
    }


def cmac_per_step(T=None):
    return ((T or ARGS_SAMPLES[0]) - (NLAGS - 1)) * NLAGS * NALPHAS * NFORMS


ARGS_SAMPLES = [T_SAMPLES]


def kernel_hash(precision, samples_per_launch=PASS):
    f = "proj_fp32.cu" if precision == "fp32" else "proj_tc.cu"
    with open(os.path.join(ROOT, "paper_2405_16911_gb300", "csrc", f), "rb") as fh:
        return f.split(".")[0] + "@" + hashlib.sha256(fh.read()).hexdigest()[:12] + "@%d" % samples_per_launch


def nvtx_range(name):
    """An NVTX range around one leg, so that a profiler can select its launches
    (`ncu --nvtx --nvtx-include "<name>/"`); a no-op where NVTX is unavailable."""
    import contextlib
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
        torch.cuda.nvtx.range_pop()
        return torch.cuda.nvtx.range(name)
    except Exception:
        return contextlib.nullcontext()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            v = [t.strip() for t in line.split(",")]
            if len(v) < 7:
                continue
            try:
                sm.append(float(v[0]))
                mx.append(float(v[1]))
            except ValueError:
                continue
            for n, flag in zip(names, v[3:7]):
                if flag.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- helpers

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def oracle_sample_rate(x, lags, alphas, target_s=10.0, max_T=1 << 16):
    """The FP64 oracle on a prefix of the stream with the full grid; GMAC/s."""
    import oracle
    M = int(np.max(lags))
    n = 256
    while True:
        t0 = time.perf_counter()
        oracle.estimate(x[:n + M], lags, alphas)
        dt = time.perf_counter() - t0
        if dt * 2 >= target_s or n >= max_T:
            break
        n = min(max_T, max(2 * n, int(n * target_s / max(dt, 1e-3) * 0.9)))
    cmac = n * len(lags) * len(alphas) * NFORMS
    return cmac / dt / 1e9, n, dt


def stored_error(R, key, T):
    """max |R - R_oracle| / R^0(0) over the sampled entries that tests/golden/bench_entries.json
    holds for workload `key` (FP64 oracle values written by make_bench_entries.py beside it);
    None when the run's stream length differs from the stored one."""
    with open(os.path.join(ROOT, "tests", "golden", "bench_entries.json")) as fh:
        g = json.load(fh)[key]
    if g["T"] != T:
        return None
    ref = np.array(g["re"]) + 1j * np.array(g["im"])
    got = R[g["form"], g["alpha_index"], g["lag_index"]]
    return float(np.max(np.abs(got - ref)) / g["r00"])


# --------------------------------------------------------------------------- serving leg

SRV_STREAMS, SRV_LAGS, SRV_ALPHAS = 256, 64, 512
SRV_CMAC_PER_SAMPLE = SRV_LAGS * SRV_ALPHAS * 2


def serving_leg(pkg, seconds=3.0, loads=(0.5, 0.9), nbase=16, blen=3 << 19):
    """Config 3: 256 streams of mixed GMSK / RRC-PSK signals, lags 0..63, 512 cycle
    frequencies, both forms, continuously batched.  Chunk lengths are log-uniform in
    [4096, 2^20]; per-stream rates are log-uniform over 100x and arrivals Poisson.  A
    saturation run measures capacity, then runs at fractions of it give submit-to-done
    latency percentiles.  Stream s draws its chunks from base signal s % 16."""
    import heapq

    import torch
    from synth import workloads
    bases = [torch.from_numpy(workloads.mix_stream(b, blen).view(np.float32)).pin_memory() for b in range(nbase)]
    lags = np.arange(SRV_LAGS)
    alphas = -0.5 + np.arange(SRV_ALPHAS) / SRV_ALPHAS
    rng = np.random.default_rng(0xC7C1_0003)
    w = 100.0 ** rng.uniform(0.0, 1.0, SRV_STREAMS)
    w /= w.sum()
    lo, hi = np.log(4096.0), np.log(float(1 << 20))
    mean_chunk = (np.exp(hi) - np.exp(lo)) / (hi - lo)
    out = {"streams": SRV_STREAMS, "lags": SRV_LAGS, "cycle_freqs": SRV_ALPHAS, "forms": 2,
           "precision": "bf16x3", "chunk": "log-uniform [4096, 1048576]", "rates": "log-uniform over 100x, Poisson"}
    with pkg.Server(max_streams=SRV_STREAMS, precision="bf16x3", ring_samples=1 << 22) as srv:
        sids = [srv.open(lags, alphas, pkg.CYC_BOTH) for _ in range(SRV_STREAMS)]
        pos = [0] * SRV_STREAMS

        def submit(i, n, tag):
            b = bases[i % nbase]
            off = pos[i] % (blen - (1 << 20))
            pos[i] += n
            srv.submit(sids[i], b.data_ptr() + 8 * off, n, tag)

        def run(rate_chunks, dur):
            """rate_chunks None: saturation (every stream always has work queued)."""
            t0 = time.perf_counter()
            done, subm, eagain, tag = [], 0, 0, 0
            events = []
            if rate_chunks is not None:
                for i in range(SRV_STREAMS):
                    heapq.heappush(events, (t0 + rng.exponential(1.0 / (rate_chunks * w[i])), i))
            b0 = srv.stats()
            while True:
                now = time.perf_counter()
                if now - t0 > dur:
                    break
                if rate_chunks is None:
                    i = int(rng.choice(SRV_STREAMS, p=w))
                else:
                    t_ev, i = events[0]
                    if t_ev > now:
                        done += srv.poll()
                        time.sleep(min(0.0005, t_ev - now))
                        continue
                    heapq.heapreplace(events, (t_ev + rng.exponential(1.0 / (rate_chunks * w[i])), i))
                n = int(np.exp(rng.uniform(lo, hi)))
                try:
                    submit(i, n, tag)
                    subm += 1
                    tag += 1
                except pkg.CycError as e:
                    if e.code != pkg.CYC_EAGAIN:
                        raise
                    eagain += 1
                    done += srv.poll()
                if tag % 64 == 0:
                    done += srv.poll()
            srv.drain(300)
            t1 = time.perf_counter()
            done += srv.poll(1 << 20)
            b1 = srv.stats()
            lat = np.array([d[5] - d[4] for d in done]) * 1e3
            nsamp = sum(d[3] for d in done)
            busy = (b1[2] - b0[2]) / 1e3
            return {"seconds": t1 - t0, "chunks": len(done), "submitted": subm, "eagain": eagain,
                    "msamples_s": nsamp / (t1 - t0) / 1e6, "gmac_s": nsamp * SRV_CMAC_PER_SAMPLE / (t1 - t0) / 1e9,
                    "gpu_busy_frac": busy / (t1 - t0), "batches": b1[0] - b0[0], "items": b1[1] - b0[1],
                    "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                    "p99_ms": float(np.percentile(lat, 99)) if lat.size else None}

        run(None, 0.5)                                   # warm-up
        sat = run(None, seconds)
        out["saturation"] = sat
        cap = sat["msamples_s"] * 1e6
        out["capacity_msamples_s"] = sat["msamples_s"]
        res = []
        for ld in loads:
            rng = np.random.default_rng(0xC7C1_0103)         # the same arrival sequence at every load
            r = run(ld * cap / mean_chunk, seconds)
            r["offered_load"] = ld
            r["offered_msamples_s"] = ld * cap / 1e6
            res.append(r)
        out["loads"] = res
    return out


def latency_leg(pkg, calls=1000, warm=20):
    """Config 0: one 65536-sample GMSK chunk (BT 0.3, 8 sps, offset 0.05, 10 dB), lags 0..31,
    64 cycle frequencies per form (k/8 CONV and 0.1 + k/8 CONJ, 8 distinct mod 1 each), FP32.
    One call = reset + push of the resident chunk on one stream per form (both queued before
    either is waited for, so the two forms' GPU work overlaps), then a read of each into host
    memory; per-call wall time percentiles over `calls` calls."""
    import torch
    from synth import workloads
    w = workloads.config0()
    x_dev = torch.from_numpy(w["x"].view(np.float32)).cuda()
    T = w["x"].size
    lags = w["lags"]
    outs = [np.empty((1, 64, 32), dtype=np.complex128) for _ in range(2)]
    torch.cuda.synchronize()
    cs = [torch.cuda.Stream(), torch.cuda.Stream()]                 # one CUDA stream per form
    with pkg.Stream(lags, w["alphas_conv"], pkg.CYC_CONV, precision="fp32", max_chunk=T,
                    cuda_stream=cs[0].cuda_stream) as sc, \
            pkg.Stream(lags, w["alphas_conj"], pkg.CYC_CONJ, precision="fp32", max_chunk=T,
                       cuda_stream=cs[1].cuda_stream) as sj:
        def call():
            for s in (sc, sj):
                s.reset()
                s.push(x_dev)
            sc.read(outs[0])
            sj.read(outs[1])
        for _ in range(warm):
            call()
        ts = []
        for _ in range(calls):
            t0 = time.perf_counter()
            call()
            ts.append(time.perf_counter() - t0)
        au = [sc.info()[1], sj.info()[1]]
        # where a call's time goes: host time to queue reset + push of both forms, the GPU
        # time of that queued work on each form's CUDA stream (events), the time the two reads
        # take after it (waiting for the GPU, the read kernel, the D2H copy, the status check),
        # and a read of an idle stream alone
        nb = max(calls // 4, 10)
        issue, gpu, rd, rd_idle = [], [], [], []
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
        for _ in range(nb):
            t0 = time.perf_counter()
            for k, s in enumerate((sc, sj)):
                ev[k][0].record(cs[k])
                s.reset()
                s.push(x_dev)
                ev[k][1].record(cs[k])
            t1 = time.perf_counter()
            sc.read(outs[0])
            sj.read(outs[1])
            t2 = time.perf_counter()
            sc.read(outs[0])
            t3 = time.perf_counter()
            issue.append(t1 - t0)
            rd.append(t2 - t1)
            rd_idle.append(t3 - t2)
            gpu.append(max(ev[0][0].elapsed_time(ev[0][1]), ev[1][0].elapsed_time(ev[1][1])) * 1e-3)
    ts = np.array(ts) * 1e6
    med = lambda v: float(np.median(np.array(v) * 1e6))
    cmac = (T - 31) * 32 * sum(au)
    return {"workload": "cfg0 GMSK 65536 samples, lags 0..31, 64 a per form (k/8: %d distinct doubles mod 1; "
                        "0.1 + k/8: %d), CONV+CONJ, fp32" % (au[0], au[1]),
            "calls": calls, "p50_us": float(np.percentile(ts, 50)), "p99_us": float(np.percentile(ts, 99)),
            "mean_us": float(ts.mean()), "gmac_s_at_p50": cmac / (np.percentile(ts, 50) * 1e-6) / 1e9,
            "call": "reset + push (device chunk) on each form's stream, then read (host) of each",
            "breakdown_median_us": {"host_issue_reset_push_both": med(issue),
                                    "gpu_reset_push_per_form_max": med(gpu),
                                    "reads_both_after_issue": med(rd), "read_idle_stream_one": med(rd_idle),
                                    "calls": nb}}


def precision_leg(pkg, reps=3):
    """Config 2: one 2^20-sample GMSK block (BT 0.5, 4 sps, 0 dB), lags 0..255, 4096 cycle
    frequencies, both forms, in each precision: device time per block (CUDA events, median
    of `reps` after one warm-up) and the error on sampled entries relative to R^0(0)."""
    import torch
    from synth import workloads
    w = workloads.config2()
    x, lags, alphas = w["x"], w["lags"], w["alphas"]
    x_dev = torch.from_numpy(x.view(np.float32)).cuda()
    T = x.size
    cmac = (T - 255) * 256 * 4096 * 2
    out = torch.empty((2, 4096, 256, 2), dtype=torch.float64, device="cuda")
    res = {"workload": "cfg2 GMSK block 2^20 samples, lags 0..255, 4096 a -0.5+k/4096, CONV+CONJ"}
    for prec in ("fp16", "bf16x3", "fp32"):
        with pkg.Stream(lags, alphas, pkg.CYC_BOTH, precision=prec, max_chunk=T) as s:
            def blk():
                s.reset()
                s.push(x_dev)
                s.read(out)
            blk()
            ms = []
            for _ in range(reps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                blk()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            R = out.cpu().numpy()
        R = R[..., 0] + 1j * R[..., 1]
        m = statistics.median(ms)
        res[prec] = {"ms": m, "gmac_s": cmac / (m * 1e-3) / 1e9, "tol": TOL[prec],
                     "err_rel_r00": stored_error(R, "cfg2", T)}
    return res


def proposer_leg(pkg, nsig=64, k=32, pushes=64):
    """Config 4: what the learned proposer buys.  One-off cost of a proposal (features, net,
    top-k, confidence) per held-out 65552-sample signal of the serving mix, and the cost of
    estimating 2^16 further samples of a stream (lags 0..63, both forms, BF16x3, pushes staged
    into 2^20-sample passes) on the full 512-point grid against the proposed cycle frequencies
    (the 2k proposals of both forms in one stream); with the recall of those proposals
    against the full-grid detections."""
    import torch
    from paper_2405_16911_gb300 import proposer_train as pt
    xs = pt.make_signals(nsig, pt.SEED_TEST)
    xd = torch.from_numpy(xs.view(np.float32)).cuda().view(nsig, pt.NS * 2)
    labels = pt.label(pkg, xd, nsig)
    net = pkg.cyc_net_create(np.load(pt.WEIGHTS), 0)
    try:
        props = [pkg.cyc_propose(net, xd[i], pt.NS, k=k) for i in range(2)]     # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        props = [pkg.cyc_propose(net, xd[i], pt.NS, k=k) for i in range(nsig)]
        t_prop = (time.perf_counter() - t0) / nsig
        rec = pt.recall_and_gain(pkg, net, xd, labels, k=k)
    finally:
        pkg.cyc_net_destroy(net)
    C = 1 << 16
    y = torch.from_numpy(np.concatenate([xs[i % nsig] for i in range(2 * pushes * C // pt.NS + 2)])[:pushes * C]
                         .view(np.float32)).cuda()

    def per_push(alphas):
        with pkg.Stream(pt.LAGS, alphas, pkg.CYC_BOTH, precision="bf16x3", max_chunk=PASS) as s:
            def run():
                s.reset()
                for c in range(pushes):
                    s.push(y[2 * c * C:2 * (c + 1) * C])
                s.sync()
            run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) * 1e-3 / pushes

    t_full = per_push(pt.GRID)
    t_top = per_push(np.concatenate([props[0][0], props[0][1]]))
    return {"workload": "cfg4 held-out serving-mix signals (65552 samples), lags 0..63, 512-point grid, "
                        "top-%d per form" % k,
            "signals": nsig, "recall": rec["recall"], "detections": rec["detections"],
            "fallback_rate": rec["fallback_rate"], "projection_work_ratio": rec["work_ratio"],
            "propose_ms_per_signal": t_prop * 1e3,
            "full_grid_us_per_2^16_samples": t_full * 1e6, "proposed_us_per_2^16_samples": t_top * 1e6,
            # a break-even length only where the proposed stream is clearly cheaper (10 %): on
            # the 512-point grid both streams are one 256-unit tile of the a-pair projection
            "breakeven_samples": (t_prop / (t_full - t_top)) * C if t_full > 1.1 * t_top else None}


def propose_timing(pkg, calls=200, nsig=8):
    """cyc_propose alone on held-out config-4 signals: wall time per call (features, net,
    top-k, confidence, the synchronisation and the copy of the proposals)."""
    import torch
    from paper_2405_16911_gb300 import proposer_train as pt
    xs = pt.make_signals(nsig, pt.SEED_TEST)
    xd = torch.from_numpy(xs.view(np.float32)).cuda().view(nsig, pt.NS * 2)
    net = pkg.cyc_net_create(np.load(pt.WEIGHTS), 0)
    try:
        for i in range(3):
            pkg.cyc_propose(net, xd[i % nsig], pt.NS, k=32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(calls):
            pkg.cyc_propose(net, xd[i % nsig], pt.NS, k=32)
        t1 = time.perf_counter()
    finally:
        pkg.cyc_net_destroy(net)
    return {"workload": "cyc_propose on held-out config-4 signals (65552 samples), top-32 per form",
            "calls": calls, "us_per_call": (t1 - t0) / calls * 1e6}


def cross_leg(pkg, x_dev, T=1 << 24, reps=2):
    """Eq. (impl-corr) in full: two inputs and signed lags at the config-1 shape -- lags
    -64..63 (128, M^- = 64), 1024 cycle frequencies, both forms, BF16x3, 2^16-sample
    pushes staged into 2^20-sample passes -- with y the config-1 stream delayed by one
    sample; device time per push next to the one-input stream (lags 0..127) on the same
    samples."""
    import torch
    C = CHUNK
    alphas = -0.5 + np.arange(NALPHAS) / NALPHAS
    y_dev = torch.roll(x_dev[:2 * T], 2)
    res = {"workload": "cfg1 shape, two inputs: lags -64..63, 1024 a, CONV+CONJ, bf16x3, %d samples" % T}
    for name, lags, cross in (("cross_signed", np.arange(-64, 64), True), ("one_input", np.arange(128), False)):
        with pkg.Stream(lags, alphas, pkg.CYC_BOTH, precision="bf16x3", max_chunk=PASS, cross=cross) as s:
            def run():
                s.reset()
                for c in range(T // C):
                    sl = slice(2 * c * C, 2 * (c + 1) * C)
                    if cross:
                        s.push(x_dev[sl], y=y_dev[sl])
                    else:
                        s.push(x_dev[sl])
                s.sync()
            run()
            ms = []
            for _ in range(reps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                run()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        m = statistics.median(ms)
        cmac = (T - 127) * 128 * NALPHAS * NFORMS
        res[name] = {"ms": m, "gmac_s": cmac / (m * 1e-3) / 1e9, "us_per_push": m * 1e3 / (T // C)}
    return res


def window_leg(pkg, x_dev, T=1 << 24, reps=2):
    """The block's windowed output (Eq. (impl-corr) at every window start k * hop, window-local
    phase) at the config-1 shape: windows of N = 65536 reference samples every 4096 samples,
    lags 0..127, 1024 cycle frequencies, both forms, BF16x3, 2^16-sample pushes staged like the
    main step's (max_chunk 2^20: a windowed stream projects up to 63 hops per pass, and every
    read of windows ends a pass), every window read into device memory after every second
    push (the ring holds 32); wall time per push next to the running-sum stream, and windows
    per second."""
    import torch
    C = CHUNK
    N, H = 1 << 16, 4096
    cap = 2 * (C // H)
    lags = np.arange(NLAGS)
    alphas = -0.5 + np.arange(NALPHAS) / NALPHAS
    out = torch.empty((cap, NFORMS, NALPHAS, NLAGS, 2), dtype=torch.float64, device="cuda")
    res = {"workload": "cfg1 shape, windows N=65536 every 4096 samples, lags 0..127, 1024 a, CONV+CONJ, bf16x3, "
                       "%d samples" % T}
    for name, window in (("windowed", (N, H, cap)), ("running_sums", None)):
        nwin = [0]
        with pkg.Stream(lags, alphas, pkg.CYC_BOTH, precision="bf16x3", max_chunk=PASS, window=window) as s:
            def run():
                s.reset()
                nwin[0] = 0
                for c in range(T // C):
                    s.push(x_dev[2 * c * C:2 * (c + 1) * C])
                    if window is not None and c % 2 == 1:       # the ring holds two pushes' windows
                        W, _ = s.read_windows(cap, out)
                        nwin[0] += W.shape[0]
                if window is not None:
                    W, _ = s.read_windows(cap, out)
                    nwin[0] += W.shape[0]
                s.sync()
            run()
            ms = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                run()
                torch.cuda.synchronize()
                ms.append((time.perf_counter() - t0) * 1e3)
        m = statistics.median(ms)
        res[name] = {"ms": m, "us_per_push": m * 1e3 / (T // C)}
        if window is not None:
            res[name]["windows"] = nwin[0]
            res[name]["windows_per_s"] = nwin[0] / (m * 1e-3)
    return res


def full_big_pushes(pkg, x_dev, out, T, CB, reps):
    """The Full-mode stream of full_leg pushed in CB-sample chunks: device ms, samples/s."""
    import torch
    with pkg.Stream(np.arange(NLAGS), None, pkg.CYC_BOTH, max_chunk=CB, full=NALPHAS) as s:
        def run_big():
            s.reset()
            for c in range(T // CB):
                s.push(x_dev[2 * c * CB:2 * (c + 1) * CB])
            s.read(out)
        run_big()
        mb = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run_big()
            e1.record()
            torch.cuda.synchronize()
            mb.append(e0.elapsed_time(e1))
    m2 = statistics.median(mb)
    return {"ms": m2, "msamples_s": T / (m2 * 1e-3) / 1e6, "us_per_push": m2 * 1e3 / (T // CB)}


def full_leg(pkg, x_dev, reps=2):
    """The paper's Full mode on the config-1 workload: every cycle frequency -1/2 + k/1024 (the
    config-1 grid itself), lags 0..127, both forms, the whole stream in 2^16-sample device
    pushes, one read at the end.  The lag products (FP32) are folded modulo 1024 in float-float
    (one launch folds up to 16 pending pushes, read in place) and one FP64 DFT per column runs
    at the read: a different algorithm from the projection, bound by shared-memory traffic
    rather than by the tensor pipe.  Reported: device time, samples/s, the direct estimator's
    complex MACs per second for the same output, the error on the stored oracle entries, and
    the same stream pushed in 2^20-sample chunks with max_chunk 2^20."""
    import torch
    C = CHUNK
    T = x_dev.numel() // 2
    out = torch.empty((NFORMS, NALPHAS, NLAGS, 2), dtype=torch.float64, device="cuda")
    with pkg.Stream(np.arange(NLAGS), None, pkg.CYC_BOTH, full=NALPHAS) as s:
        def run():
            s.reset()
            for c in range(T // C):
                s.push(x_dev[2 * c * C:2 * (c + 1) * C])
            s.read(out)
        run()
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        R = out.cpu().numpy()
        # f4: cyclic spectra of that estimate, 256 frequencies, Hann lag window
        spec = torch.empty((NFORMS, NALPHAS, 256, 2), dtype=torch.float64, device="cuda")
        s.read_spectrum(256, 1, spec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            s.read_spectrum(256, 1, spec)
        t_spec = (time.perf_counter() - t0) / 5
    m = statistics.median(ms)
    R = R[..., 0] + 1j * R[..., 1]
    CB = 1 << 20
    big = None
    if T >= 4 * CB:
        big = full_big_pushes(pkg, x_dev, out, T, CB, reps)
    return {"spectrum_ms": t_spec * 1e3,
            "pushes_2^20": big,
            "windows": full_windows(pkg, x_dev, min(T, 1 << 24), reps),
            "spectrum": "cyc_read_spectrum: 2 x 1024 cycle frequencies x 256 frequencies over 128 lags, Hann, FP64",
            "workload": "cfg1 stream, Full mode: a = -0.5 + k/1024 by folding mod 1024, lags 0..127, CONV+CONJ, "
                        "%d samples in 2^16 pushes, fp32 products, float-float fold, fp64 DFT" % T,
            "ms": m, "msamples_s": T / (m * 1e-3) / 1e6, "us_per_push": m * 1e3 / (T // C),
            "direct_equivalent_gmac_s": cmac_per_step(T) / (m * 1e-3) / 1e9,
            "err_rel_r00": stored_error(R, "cfg1", T), "err_tol": TOL["fp32"]}


def full_windows(pkg, x_dev, T, reps):
    """Full mode per window (Sec. 4 Full mode: every a = -1/2 + k/N of each window by one
    N-point FFT per lag, window-local phase) at the config-1 shape: windows of N = 1024
    reference samples every 1024 samples, lags 0..127, both forms, 2^16-sample device pushes
    (64 windows each), every window read into device memory after every second push.  Each
    window is 2 x 1024 x 128 complex values: 2 MB in the FP32 ring, 4 MB read out in FP64, so
    the mode is bound by writing and reading those (8 MB of HBM traffic per window)."""
    import torch
    C = CHUNK
    A = H = NALPHAS
    cap = 2 * (C // H)
    out = torch.empty((cap, NFORMS, A, NLAGS, 2), dtype=torch.float64, device="cuda")
    nwin = [0]
    with pkg.Stream(np.arange(NLAGS), None, pkg.CYC_BOTH, full=A, window=(A, H, cap)) as s:
        def run():
            s.reset()
            nwin[0] = 0
            for c in range(T // C):
                s.push(x_dev[2 * c * C:2 * (c + 1) * C])
                if c % 2 == 1:
                    W, _ = s.read_windows(cap, out)
                    nwin[0] += W.shape[0]
            W, _ = s.read_windows(cap, out)
            nwin[0] += W.shape[0]
            s.sync()
        run()
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    m = statistics.median(ms)
    win_bytes = NFORMS * A * NLAGS * (8 + 8 + 16)          # ring write, ring read, FP64 out
    return {"workload": "Full mode per window: N = 1024 every 1024 samples, lags 0..127, CONV+CONJ, "
                        "%d samples in 2^16 pushes, windows read into device memory every second push" % T,
            "ms": m, "us_per_push": m * 1e3 / (T // C), "windows": nwin[0],
            "windows_per_s": nwin[0] / (m * 1e-3),
            "ring_and_out_gb_s": nwin[0] * win_bytes / (m * 1e-3) / 1e9}


# --------------------------------------------------------------------------- reference arm

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from synth import workloads
    oracle.build()
    T_s = 4096
    w = workloads.config1(T=T_s + NLAGS - 1)
    x, lags, alphas = w["x"], w["lags"], w["alphas"]
    for _ in range(args.warmup):
        oracle.estimate(x, lags, alphas)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.estimate(x, lags, alphas)
    dt = (time.perf_counter() - t0) / args.steps
    cmac = T_s * NLAGS * NALPHAS * NFORMS
    v = cmac / dt / 1e9
    cores = oracle.max_threads()
    sample = "first %d committed samples of the config-1 stream, full grid (1024 a x 128 lags x 2 forms)" % T_s
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config("fp64 oracle"),
        "msamples_per_s": T_s / dt / 1e6,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- our arm

def time_device_steps(pkg, x_dev, lags, alphas, precision, steps, warmup, world, profile, n0=0, merge=False):
    """Steps over the device-resident samples x_dev (pushes of CHUNK samples, the last one
    possibly shorter); merge=True: the ranks hold time shards of one stream (start index
    n0), merged by one in-place all-reduce of the running sums before the read."""
    import torch
    from paper_2405_16911_gb300 import shard
    out = torch.empty((NFORMS, NALPHAS, NLAGS, 2), dtype=torch.float64, device="cuda")
    nsamp = x_dev.numel() // 2
    with pkg.Stream(lags, alphas, pkg.CYC_BOTH, precision=precision, max_chunk=PASS, n0=n0) as s:
        def step():
            s.reset()
            for c0 in range(0, nsamp, CHUNK):
                s.push(x_dev[2 * c0:2 * min(c0 + CHUNK, nsamp)])
            if merge:
                shard.allreduce_stream(s)
            s.read(out)
        for _ in range(warmup):
            step()
        s.profile(profile)
        s.profile_read()
        barrier(world)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
        barrier(world)
        ms = ev0.elapsed_time(ev1) / steps
        proj_ms, proj_launches, kernels = s.profile_read()
        R = out.cpu().numpy()
    return ms, R[..., 0] + 1j * R[..., 1], proj_ms, proj_launches, kernels


def time_e2e(pkg, x_host_pinned, lags, alphas, precision, steps):
    """Host buffers through the public API: H2D of every chunk and D2H of the result inside."""
    nchunks = x_host_pinned.numel() // (2 * CHUNK)
    res = np.empty((NFORMS, NALPHAS, NLAGS), dtype=np.complex128)
    base = x_host_pinned.data_ptr()
    with pkg.Stream(lags, alphas, pkg.CYC_BOTH, precision=precision, max_chunk=PASS) as s:
        def step():
            s.reset()
            for c in range(nchunks):
                s.push(base + c * CHUNK * 8, CHUNK, 0)
            s.read(res)
        step()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        dt = (time.perf_counter() - t0) / steps
    return dt, x_host_pinned.numel() * 4, res.nbytes


def run_ours(args):
    import torch

    import paper_2405_16911_gb300 as pkg
    from synth import workloads

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    pkg.load()
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None else None
    precision = args.precision
    try:
        pkg.Stream([0], [0.0], pkg.CYC_BOTH, precision=precision).close()
    except pkg.CycError as e:
        if e.code != pkg.CYC_ENOTSUP:
            raise
        precision = "fp32"

    sharded = args.shard and world > 1
    w = workloads.config1(T=args.samples, replica=0 if sharded else rank)
    x, lags, alphas = w["x"], w["lags"], w["alphas"]
    n0 = 0
    if sharded:
        # one stream of T samples cut into time shards, one per rank (strong scaling)
        from paper_2405_16911_gb300 import shard
        s0, s1, n0, _ = shard.time_shards(x.size, NLAGS - 1, world)[rank]
        x_dev = torch.from_numpy(np.ascontiguousarray(x[s0:s1]).view(np.float32)).cuda()
    else:
        x_dev = torch.from_numpy(x.view(np.float32)).cuda()

    sampler = ClockSampler(uuid)
    ms, R, proj_ms, proj_launches, kernels = time_device_steps(
        pkg, x_dev, lags, alphas, precision, args.steps, args.warmup, world, True, n0=n0, merge=sharded)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, world)
    cmac = cmac_per_step() * (1 if sharded else world)
    value = cmac / (ms * 1e-3) / 1e9

    # roofline of the projection kernel (the dominant kernel of the step)
    nsm = props.multi_processor_count
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    cmac_launch = cmac_per_step() / (world if sharded else 1) * args.steps / max(proj_launches, 1)
    avg_launch_s = proj_ms * 1e-3 / max(proj_launches, 1)
    if precision == "fp32":
        clk = float(peaks.get("sm_max_mhz", 2070.0))
        peak = nsm * 128 * 2 * clk * 1e6 / 1e12
        achieved = cmac_launch * FLOPS_PER_CMAC / avg_launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "FP32 FMA pipes: %d SMs x 128 lanes x 2 flop x %.0f MHz (max SM clock)" % (nsm, clk)}
    else:
        passes = TC_PASSES[precision]
        if "bf16_tflops_sustained" in peaks:
            peak, src = float(peaks["bf16_tflops_sustained"]), "measured bf16 sustained (MEASURED_PEAKS.json)"
        else:
            peak, src = 1700.0, "fallback bf16 sustained"
        # achieved: algorithmic flops (8 per CMAC); executed: what the tensor pipe ran
        achieved = cmac_launch * FLOPS_PER_CMAC / avg_launch_s / 1e12
        fexec = TC_EXEC_FLOPS_PER_CMAC_PASS * passes
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "peak_source": src,
                "flops_per_cmac": FLOPS_PER_CMAC, "executed_flops_per_cmac": fexec,
                "executed_tflops": cmac_launch * fexec / avg_launch_s / 1e12}
        roof["executed_frac"] = roof["executed_tflops"] / peak
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC.get(kernel_hash(precision))
    roof["kernel_ms_avg"] = avg_launch_s * 1e3
    roof["share_of_step"] = proj_ms / args.steps / ms

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16", "fp16": "f16"}[precision],
        "data": "synthetic", "config": workload_config(precision),
        "msamples_per_s": ARGS_SAMPLES[0] * (1 if sharded else world) / (ms * 1e-3) / 1e6,
        "precision": {"fp32": "fp32 CUDA-core projection", "bf16x3": "bf16 hi/lo split, 3 products, fp32 accumulate",
                      "fp16": "fp16 single pass, fp32 accumulate"}[precision] + "; fp64 running sums",
        "gpu_launches": kernels, "roofline": roof, "clocks": clocks,
    }
    if rank == 0:
        line["err_rel_r00"] = stored_error(R, "cfg1", ARGS_SAMPLES[0])
        line["err_tol"] = TOL[precision]

    if rank == 0 and not args.no_e2e:
        xh = torch.from_numpy(x.view(np.float32)).pin_memory()
        dt, hb, db = time_e2e(pkg, xh, lags, alphas, precision, max(1, min(args.steps, 3)))
        line["e2e"] = {"value": cmac_per_step() / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": hb,
                       "d2h_bytes_per_step": db, "ms_per_step": dt * 1e3,
                       "path": "cyc_push from page-locked host memory, cyc_read into host memory"}
        del xh
    if rank == 0 and precision != "fp32" and not args.no_plain:
        k = max(1, min(args.steps, 2))
        ms32, R32, pms, pl, _ = time_device_steps(pkg, x_dev, lags, alphas, "fp32", k, 1, 1, True)
        line["plain_fp32"] = {"value": cmac_per_step() / (ms32 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms32,
                              "steps": k, "err_rel_r00": stored_error(R32, "cfg1", ARGS_SAMPLES[0])}
        line["speedup_vs_plain_fp32"] = value / world / line["plain_fp32"]["value"]
    if rank == 0 and not args.no_serving:
        with nvtx_range("serving"):
            line["serving"] = serving_leg(pkg, seconds=args.serving_seconds)
        line["p99_ms"] = line["serving"]["loads"][-1]["p99_ms"]
    if rank == 0 and not args.no_latency:
        with nvtx_range("cfg0_latency"):
            line["cfg0_latency"] = latency_leg(pkg)
    if rank == 0 and not args.no_precisions:
        with nvtx_range("cfg2_precisions"):
            line["cfg2_precisions"] = precision_leg(pkg)
    if rank == 0 and not args.no_cross:
        with nvtx_range("f1_cross"):
            line["f1_cross"] = cross_leg(pkg, x_dev, T=min(1 << 24, ARGS_SAMPLES[0]))
    if rank == 0 and not args.no_full:
        with nvtx_range("f3_full_mode"):
            line["f3_full_mode"] = full_leg(pkg, x_dev)
    if rank == 0 and not args.no_windows:
        with nvtx_range("f2_windows"):
            line["f2_windows"] = window_leg(pkg, x_dev, T=min(1 << 24, ARGS_SAMPLES[0]))
    if rank == 0 and not args.no_proposer:
        with nvtx_range("cfg4_proposer"):
            line["cfg4_proposer"] = proposer_leg(pkg)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        v, n, dt = oracle_sample_rate(x, lags, alphas, target_s=args.cpu_seconds)
        n1 = max(256, n // 16)
        t0 = time.perf_counter()
        oracle.estimate(x[:n1 + int(np.max(lags))], lags, alphas, threads=1)
        v1 = n1 * len(lags) * len(alphas) * NFORMS / (time.perf_counter() - t0) / 1e9
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                                "sample": "first %d committed samples of the stream, full grid "
                                          "(1024 a x 128 lags x 2 forms), %.1f s" % (n, dt),
                                "value_1core": v1, "sample_1core": "first %d committed samples, one thread" % n1,
                                "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16x3", "fp16", "fp32"], default="bf16x3")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-seconds", type=float, default=3.0)
    ap.add_argument("--no-latency", action="store_true", help="skip the config-0 per-call latency leg")
    ap.add_argument("--no-precisions", action="store_true", help="skip the config-2 precision leg")
    ap.add_argument("--no-proposer", action="store_true", help="skip the config-4 proposer leg")
    ap.add_argument("--no-cross", action="store_true", help="skip the two-input / signed-lag leg")
    ap.add_argument("--no-windows", action="store_true", help="skip the windowed-output leg")
    ap.add_argument("--no-full", action="store_true", help="skip the Full-mode leg")
    ap.add_argument("--serving-only", action="store_true", help="run the serving leg alone and print it")
    ap.add_argument("--latency-only", action="store_true", help="run the config-0 latency leg alone and print it")
    ap.add_argument("--latency-calls", type=int, default=1000)
    ap.add_argument("--propose-only", action="store_true", help="time cyc_propose alone and print it")
    ap.add_argument("--propose-calls", type=int, default=200)
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1 ranks: cut one config-1 stream into N time shards and merge them with one "
                         "all-reduce of the running sums (strong scaling) instead of N independent replicas")
    ap.add_argument("--samples", type=int, default=T_SAMPLES,
                    help="stream length per step (multiple of 2^16); smaller values only for profiling")
    args = ap.parse_args()
    if args.samples % CHUNK or args.samples < CHUNK:
        ap.error("--samples must be a positive multiple of %d" % CHUNK)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    ARGS_SAMPLES[0] = args.samples
    if args.serving_only:
        import torch
        import paper_2405_16911_gb300 as pkg
        torch.cuda.set_device(0)
        pkg.load()
        print(json.dumps(serving_leg(pkg, seconds=args.serving_seconds)))
        return 0
    if args.propose_only:
        import torch
        import paper_2405_16911_gb300 as pkg
        torch.cuda.set_device(0)
        pkg.load()
        print(json.dumps(propose_timing(pkg, calls=args.propose_calls)))
        return 0
    if args.latency_only:
        import torch
        import paper_2405_16911_gb300 as pkg
        torch.cuda.set_device(0)
        pkg.load()
        with nvtx_range("latency"):
            print(json.dumps(latency_leg(pkg, calls=args.latency_calls)))
        return 0
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
