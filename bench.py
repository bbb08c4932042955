"""Benchmark of the xorgens GPU path (one JSON line on stdout).

Step = one pass of the generation hot path over the many-streams workload:
16384 streams (seeds 1..16384), 2^16 u32 words per stream (2^30 words, 4 GiB)
then 2^16 FP32 uniforms per stream (another 4 GiB), with the stream state
resident in HBM and advancing from step to step.  value = RN/s over the timed
steps (CUDA events on the launching stream, max over ranks).  The outputs
(8 GiB per step) are far larger than L2 (129 MB), so no flush is needed.

Beside the headline it reports the same metric end to end through the C ABI
into pinned host memory (e2e), the roofline of the dominant kernel against
the measured HBM peak, per-row figures (normals, fused sum), the SM clocks
seen during the timed region, and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 and no WORLD_SIZE in the environment the script starts N
ranks of itself (one per GPU) through torch's launcher; under an external
launcher it runs as the rank it is given.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1108_0486_gb300 import workloads as W  # noqa: E402

STREAMS = W.MANY_STREAMS["streams"]
N_PER = W.MANY_STREAMS["n"]
WORKLOAD = ("16384 streams (seeds 1..16384), 2^16 u32 + 2^16 FP32 uniforms per stream "
            "per step (2^31 RNs, 8 GiB written); xorgens (r,s,a,b,c,d)=(128,95,17,12,13,15), Weyl on")
CONFIG = {"workload": WORKLOAD, "streams": STREAMS, "n_per_stream": N_PER,
          "outputs": ["u32", "uniform_f32"], "param_set": "(128,95,17,12,13,15)",
          "l2_flush": "none needed: 8 GiB of outputs per step >> 129 MB L2"}
METRIC, UNIT = "RN/s", "RN/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _fp8_peak():
    """Dense FP8 tensor peak: the measured bf16 GEMM rate times the nominal
    FP8 / bf16 ratio of 2, else the nominal 4.5 PFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return 2.0 * float(json.load(f)["bf16_tflops"]), "measured bf16 x 2"
    except Exception:
        return 4500.0, "nominal"


def _record(name):
    """A profiles/ record (key value lines) taken with ncu, if it was taken
    on the current kernel sources (else None)."""
    import hashlib
    try:
        rec = {}
        for line in open(os.path.join(ROOT, "profiles", name)):
            if line.strip() and not line.startswith("#"):
                k, v = line.split(None, 1)
                rec[k] = v.strip()
        src = b"".join(open(os.path.join(ROOT, "paper_1108_0486_gb300", "csrc", f), "rb").read()
                       for f in ("xg_device.cuh", "xg_kernels.cuh"))
        if hashlib.sha256(src).hexdigest()[:16] != rec.get("kernel_sources_sha256_16"):
            return None
        return rec
    except Exception:
        return None


def _traffic(kernel=None):
    """ncu DRAM bytes per launch of the dominant kernel, if recorded for the
    current kernel sources (else None)."""
    rec = _record("gen_kernel_traffic.txt")
    if rec is None or (kernel is not None and rec.get("kernel") != kernel):
        return None
    return float(rec["traffic_bytes_per_launch"])


def _issue_ceiling(sm_count, sm_mhz):
    """Normals per second at full instruction issue (4 warp instructions per
    SM per clock) for the recorded instruction count of gen_kernel<normal>,
    or None when the record does not match the kernel sources."""
    rec = _record("gen_kernel_normal_issue.txt")
    if rec is None or not sm_mhz:
        return None
    per_normal = float(rec["warp_instructions"]) / float(rec["normals"])
    return {"normals_per_s": sm_count * 4 * sm_mhz * 1e6 / per_normal,
            "instructions_per_normal": round(32 * per_normal, 2), "sm_mhz": sm_mhz,
            "source": "profiles/gen_kernel_normal_issue.txt (ncu smsp__inst_executed.sum, 16384 x 4096 case)"}


def _free_port() -> int:
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(n: int, argv) -> int:
    """Run this script as n ranks on one node, one per GPU (torch's elastic
    launcher, rendezvous on 127.0.0.1): each rank reads RANK, LOCAL_RANK and
    WORLD_SIZE from its environment and rank 0 prints the line.  Returns the
    launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__),
           *argv]
    return subprocess.call(cmd)


def rank_check(args):
    """Launcher check without GPU work (not a bench line): every rank joins a
    gloo group, reports its stream seeds, and rank 0 prints the ranks seen
    and the slowest rank's time, each rank having taken 1 + rank ms."""
    import torch.distributed as dist
    ws, rank, _ = _dist()
    dist.init_process_group("gloo")
    seeds = rank_seeds(rank)
    gathered = [None] * ws
    dist.all_gather_object(gathered, (rank, int(seeds[0]), int(seeds[-1]), int(seeds.size)))
    ms = max_over_ranks(1.0 + rank, dist, "cpu")
    if rank == 0:
        print(json.dumps({"rank_check": True, "n_gpus": ws, "requested": args.gpus, "ranks": gathered,
                          "max_ms": ms}), flush=True)
    dist.barrier()
    dist.destroy_process_group()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seeds(rank: int):
    """Weak scaling: every rank owns its own 16384 streams, seeded with
    consecutive integers that no other rank uses."""
    return W.seeds(STREAMS, start=1 + rank * STREAMS)


def max_over_ranks(ms: float, dist, device) -> float:
    """The job's time is the slowest rank's (no data-path collective: the
    streams are independent; only the timing is reduced)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- oracle

def cpu_baseline(target_s: float = 10.0):
    """The CPU oracle as it stands, threaded over streams on every host core
    (ctypes releases the GIL), on a sample of the workload's streams."""
    import oracle as O
    cores = os.cpu_count() or 1
    O.lib()

    def run(seed_list):
        threads = []
        parts = np.array_split(seed_list, cores)
        for p in parts:
            if p.size == 0:
                continue
            def job(p=p):
                O.streams(p, N_PER, kind="u32")
                O.streams(p, N_PER, kind="uniform")
            threads.append(threading.Thread(target=job))
        t0 = time.perf_counter()
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        return time.perf_counter() - t0

    probe = W.seeds(cores * 2)
    dt = run(probe)
    per_stream = dt / probe.size
    n_streams = int(min(STREAMS, max(cores, target_s / max(per_stream, 1e-9))))
    sample = W.seeds(n_streams)
    passes, dt = 0, 0.0
    while dt < target_s and passes < 64:
        dt += run(sample)
        passes += 1
    rns = passes * n_streams * 2 * N_PER / dt
    return {"value": rns, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} pass(es) over {n_streams} of the 16384 streams, 2^16 u32 + 2^16 "
                      f"uniforms each ({passes * n_streams * 2 * N_PER} RNs, {dt:.1f} s wall on "
                      f"{cores} threads)"}


def _threaded(jobs, cores):
    """Run the callables in `jobs` on `cores` threads (ctypes releases the
    GIL inside the oracle); returns the wall time."""
    parts = [jobs[i::cores] for i in range(cores)]
    threads = [threading.Thread(target=lambda p=p: [j() for j in p]) for p in parts if p]
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return time.perf_counter() - t0


def _oracle_draw(g, kind, count, chunk=1 << 22):
    """count outputs of kind 0 u32 / 1 uniform / 2 normal (FP64) from oracle
    generator g, in chunks (even, so normal pairs stay aligned)."""
    fn = (g.u32, g.uniform, g.normal64)[kind]
    while count > 0:
        m = min(count, chunk)
        fn(m)
        count -= m


def oracle_row_baselines(target_s: float = 4.0):
    """The CPU oracle as it stands on the other rows' workloads, each on a
    bounded sample: c0 one stream of 2^20 words on one thread; the 2^30
    normals (FP64 oracle) and the uneven batch threaded over streams / items;
    a 1% sample of the serving requests, each drawn from its stream's fresh
    seed, threaded over requests."""
    import oracle as O
    O.lib()
    cores = os.cpu_count() or 1
    out = {}
    # c0: single stream, single thread, the whole workload
    g = O.Xorgens.param_set(0).seed(W.SINGLE_STREAM["seed"])
    t0 = time.perf_counter()
    g.u32(W.SINGLE_STREAM["n"])
    dt = time.perf_counter() - t0
    out["single_stream_2p20_u32"] = {"value": W.SINGLE_STREAM["n"] / dt, "unit": UNIT, "cores": 1,
                                     "kind": "oracle", "sample": "the whole workload: one stream, 2^20 u32"}
    # c2: FP64 normals, 2^16 per stream, threaded over a sample of streams
    n = W.NORMALS["n"]
    probe = time.perf_counter()
    O.streams(W.seeds(1), n, kind="normal")
    per_stream = time.perf_counter() - probe
    k = int(min(W.NORMALS["streams"], max(cores, cores * target_s / max(per_stream, 1e-6))))
    seeds = W.seeds(k)
    dt = _threaded([lambda s=s: O.streams(seeds[s:s + 1], n, kind="normal") for s in range(k)], cores)
    out["normal"] = {"value": k * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                     "sample": f"{k} of the 16384 streams x 2^16 FP64 normals ({dt:.1f} s wall)"}
    # c3: the uneven batch, threaded over items; every m-th item
    items = W.batched_uneven()
    total = sum(it.count for it in items)
    rate = k * n / dt * 1.5  # rough mixed-type rate, only to size the sample
    m = max(1, int(np.ceil(total / (rate * target_s))))
    pick = items[::m]
    words = sum(it.count for it in pick)
    jobs = [lambda it=it: _oracle_draw(O.Xorgens.param_set(0).seed(it.stream + 1), it.kind, it.count)
            for it in pick]
    dt = _threaded(jobs, cores)
    out["batched"] = {"value": words / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                      "sample": f"1 in {m} of the 4096 items ({len(pick)} items, {words} outputs, "
                                f"{dt:.1f} s wall)"}
    # c4: a 1% sample of the 10 s serving requests
    all_reqs = W.serving_requests(n_streams=65536, rate=20000.0, duration=10.0)
    reqs = all_reqs[::100]
    words = sum(r.count for r in reqs)
    jobs = [lambda r=r: _oracle_draw(O.Xorgens.param_set(0).seed(r.stream + 1), r.kind, r.count)
            for r in reqs]
    dt = _threaded(jobs, cores)
    out["serving"] = {"value": words / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                      "sample": f"1 in 100 of the {len(all_reqs)} requests ({len(reqs)} requests, "
                                f"{words} outputs, each from its stream's fresh seed; {dt:.1f} s wall)"}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    O.lib()
    cores = os.cpu_count() or 1
    base = cpu_baseline(target_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)))
    n_streams = int(base["sample"].split(" over ")[1].split(" of ")[0])
    sample = W.seeds(n_streams)

    def step():
        parts = np.array_split(sample, cores)
        th = []
        for p in parts:
            if p.size:
                th.append(threading.Thread(target=lambda p=p: (O.streams(p, N_PER, kind="u32"),
                                                               O.streams(p, N_PER, kind="uniform"))))
        for t in th:
            t.start()
        for t in th:
            t.join()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    rns = n_streams * 2 * N_PER * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": rns, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": rns, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {n_streams} of the 16384 streams, "
                                       "2^16 u32 + 2^16 uniforms each"},
            "e2e": {"value": rns, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1108_0486_gb300 import Streams, _lib as L

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # weak scaling: every rank owns its own 16384 streams (seeds offset by rank)
    seeds = rank_seeds(rank)
    st = Streams(STREAMS, seeds=seeds, stream=stream)
    buf_u = torch.empty((STREAMS, N_PER), dtype=torch.int32, device="cuda")
    buf_f = torch.empty((STREAMS, N_PER), dtype=torch.float32, device="cuda")
    launches_per_step = 2
    tuned = {}
    if not args.no_autotune:
        for kind in ("u32", "uniform", "normal"):
            tuned[kind] = st.autotune(kind, N_PER)

    ev = []  # (start, mid, end) events per step: u32 kernel, uniform kernel

    def step(record=False):
        if record:
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            st.u32(N_PER, out=buf_u)
            e1.record(stream)
            st.uniform(N_PER, out=buf_f)
            e2.record(stream)
            ev.append((e0, e1, e2))
        else:
            st.u32(N_PER, out=buf_u)
            st.uniform(N_PER, out=buf_f)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def timed_region():
        ev.clear()
        if dist:
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t_start.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t_end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = t_start.elapsed_time(t_end)
        return max_over_ranks(ms, dist, "cuda"), clocks.stop()

    ms, clk = timed_region()
    if _throttled(clk, dist):
        # a clock record with a slowdown (or clocks well below their maximum
        # for no reason) is measured once more; both records are reported
        first = {"ms": ms, "clocks": clk}
        ms, clk = timed_region()
        clk = dict(clk, remeasured_after=first)
    ms_u = [a.elapsed_time(b) for a, b, _ in ev]
    ms_f = [b.elapsed_time(c) for _, b, c in ev]
    rns_per_step = STREAMS * N_PER * 2
    value = rns_per_step * args.steps * ws / (ms / 1e3)
    peak, peak_kind = _peaks()
    bytes_per_launch = STREAMS * N_PER * 4
    avg_u = sum(ms_u) / len(ms_u)
    avg_f = sum(ms_f) / len(ms_f)
    dom_ms, dom_name = (avg_u, "gen_kernel<u32>") if avg_u >= avg_f else (avg_f, "gen_kernel_ilp<uniform>")
    achieved = bytes_per_launch / (dom_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": args.traffic if args.traffic is not None else _traffic(dom_name),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "per_kernel_ms": {"u32": avg_u, "uniform": avg_f}}
    # context for a write-only kernel: a memset-style write of the same
    # size (torch's zero_ of the step's u32 buffer, best of five), measured here
    wbest = min(_time(lambda: buf_u.zero_(), stream, torch, reps=1, warm=1) for _ in range(5))
    write_gbs = bytes_per_launch / (wbest / 1e3) / 1e9
    roofline["write_only_reference"] = {"gbs": write_gbs, "how": "torch zero_ of 4 GiB, best of 5",
                                        "frac_of_it": achieved / write_gbs}

    # the end-to-end figure right after the headline, on the same streams,
    # before the other rows run
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(st, stream, torch, L, args, dist, ws)
    rows = {}
    if not args.quick and rank == 0:
        # the other rows run on one GPU (with N > 1 the other ranks wait)
        rows = extra_rows(st, stream, torch, peak, sm_mhz=clk.get("sm_mhz") or clk.get("sm_max_mhz"))
        rows["batched"] = batched_row(torch, L, stream, peak)
        rows["serving"] = serving_row(torch, L, stream, seconds=args.serve_seconds)
        rows["serving_sweep"] = serving_sweep(torch, L, stream)
        rows["serving_sweep_u32_uniform"] = serving_sweep_words(torch, L, stream, peak)
        try:
            rows["curand_xorwow_context"] = curand_row(torch, stream)
        except Exception as e:  # context only: never fail the bench on it
            rows["curand_xorwow_context"] = {"unavailable": str(e)[:200]}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    st.close()
    del buf_u, buf_f
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": dict(CONFIG, parallelism=f"independent streams x{ws}", launch=tuned),
                "roofline": roofline, "gpu_launches": launches_per_step * args.steps * ws,
                "clocks": clk, "e2e": e2e, "rows": rows}
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline()
            if rows:
                for name, base in oracle_row_baselines().items():
                    if isinstance(rows.get(name), dict):
                        rows[name]["cpu_baseline"] = base
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _throttled(clk, dist=None) -> bool:
    """A slowdown reason, or a median SM clock below 90% of its maximum with
    no reason given, on any rank."""
    bad = bool(set(clk.get("reasons", [])) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"})
    sm, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and mx and sm < 0.9 * mx and not clk.get("reasons"):
        bad = True
    if dist:
        import torch
        t = torch.tensor([1.0 if bad else 0.0], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        bad = bool(t.item())
    return bad


def _time(fn, stream, torch, reps=5, warm=2):
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sum(ts) / len(ts)


def extra_rows(st, stream, torch, peak, sm_mhz=None):
    """Other rows of the path on the same streams: normals (2^30 FP32 over
    16384 streams) and the fused normal sum (no bulk HBM write).  The normal
    row also reports its issue ceiling: normals are instruction-bound."""
    rows = {}
    n = W.NORMALS["n"]
    buf = torch.empty((STREAMS, n), dtype=torch.float32, device="cuda")
    ms = _time(lambda: st.normal(n, out=buf), stream, torch)
    rn = STREAMS * n
    rows["normal"] = {"rn_s": rn / (ms / 1e3), "ms": ms,
                      "hbm_frac": rn * 4 / (ms / 1e3) / 1e9 / peak, "launch": st.get_launch("normal")}
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    ceil = _issue_ceiling(sm_count, sm_mhz)
    if ceil is not None and tuple(rows["normal"]["launch"]) == (32, 2):
        ceil["frac"] = rows["normal"]["rn_s"] / ceil["normals_per_s"]
        rows["normal"]["issue_ceiling"] = ceil
    sums = torch.empty(STREAMS, dtype=torch.float32, device="cuda")
    ms = _time(lambda: st.normal_sum(n, out=sums), stream, torch)
    rows["normal_sum_fused"] = {"rn_s": rn / (ms / 1e3), "ms": ms, "hbm_bytes_written": STREAMS * 4}
    ms = _time(lambda: st.u32(n, out=buf.view(torch.int32)), stream, torch)
    rows["u32"] = {"rn_s": rn / (ms / 1e3), "ms": ms, "hbm_frac": rn * 4 / (ms / 1e3) / 1e9 / peak}
    # the paper's parameter set (128,65,15,14,12,17) on the same kernels,
    # its own autotuned launch shapes: 2^16 u32 and 2^16 uniforms per stream
    from paper_1108_0486_gb300 import Streams as _S
    sp = _S(STREAMS, param_set=1, seeds=W.seeds(STREAMS), stream=stream)
    paper = {"param_set": "(128,65,15,14,12,17)", "launch": {}}
    for kind in ("u32", "uniform"):
        paper["launch"][kind] = sp.autotune(kind, n)
        view = buf.view(torch.int32) if kind == "u32" else buf
        msk = _time(lambda: sp.generate(kind, n, out=view), stream, torch)
        paper[kind] = {"ms": msk, "rn_s": rn / (msk / 1e3), "hbm_frac": rn * 4 / (msk / 1e3) / 1e9 / peak}
    sp.close()
    rows["paper_parameter_set"] = paper
    del buf
    # jump-ahead of every stream: J = 2^40 + 2^20 + 12345 words, 8 set bits,
    # i.e. 8 applications of a 4096 x 4096 GF(2) matrix per stream
    J = (1 << 40) + (1 << 20) + 12345
    ms = _time(lambda: st.jump(J), stream, torch)
    bits = bin(J).count("1")
    # the powers are multiplied first ((bits - 1) applications to the 4096
    # columns of a matrix), then the product is applied to the streams; each
    # application of a 4096 x 4096 GF(2) matrix to one state is 2 * 4096^2
    # FP8 tensor operations on the tensor-core path
    apps = (bits - 1) * 4096 + STREAMS
    tflops = 2 * 4096 ** 2 * apps / (ms / 1e3) / 1e12
    fp8_peak = _fp8_peak()
    os.environ["XG_JUMP_TENSOR_CORES"] = "0"
    try:
        ms_table = _time(lambda: st.jump(J), stream, torch)
    finally:
        del os.environ["XG_JUMP_TENSOR_CORES"]
    rows["jump_16384_streams"] = {"words": J, "set_bits": bits, "ms": ms, "state_applications": apps,
                                  "tensor_tflops": tflops, "fp8_peak_tflops": fp8_peak[0],
                                  "fp8_peak_source": fp8_peak[1], "frac_of_fp8_peak": tflops / fp8_peak[0],
                                  "ms_table_kernel": ms_table,
                                  "note": "whole call: gather, FP8 expansion, tensor-core GEMMs, scatter"}
    # 16384 disjoint substreams of one sequence, 2^40 words apart (14 doubling
    # steps, one matrix application per stream); the streams are re-seeded
    # with their own seeds afterwards
    ms = _time(lambda: st.seed_substreams(1, 40), stream, torch)
    rows["seed_substreams_16384_streams"] = {"log2_spacing": 40, "ms": ms}
    st.seed(W.seeds(STREAMS))
    # one stream, 2^20 words (seed 0x12345678): latency of a single long call
    from paper_1108_0486_gb300 import Streams
    one = Streams(1, seeds=[W.SINGLE_STREAM["seed"]], stream=stream)
    nb = W.SINGLE_STREAM["n"]
    ob = torch.empty(nb, dtype=torch.int32, device="cuda")
    ms_cut = _time(lambda: one.u32(nb, out=ob.view(1, nb)), stream, torch)
    one.set_batch_split(1)
    ms_serial = _time(lambda: one.u32(nb, out=ob.view(1, nb)), stream, torch)
    one.close()
    rows["single_stream_2p20_u32"] = {"ms": ms_cut, "rn_s": nb / (ms_cut / 1e3),
                                      "ms_one_warp_uncut": ms_serial}
    # 64-bit words: 16384 streams x 2^16 FP64 uniforms (8 GiB) and raw u64
    from paper_1108_0486_gb300 import Streams64
    s64 = Streams64(STREAMS, seeds=W.seeds(STREAMS), stream=stream)
    n64 = N_PER
    b64 = torch.empty((STREAMS, n64), dtype=torch.float64, device="cuda")
    tuned64 = s64.autotune("uniform", n64)
    tuned64u = s64.autotune("u64", n64)
    ms_f = _time(lambda: s64.uniform(n64, out=b64), stream, torch)
    ms_u = _time(lambda: s64.u64(n64, out=b64.view(torch.int64)), stream, torch)
    rn64 = STREAMS * n64
    rows["w64_uniform_f64"] = {"rn_s": rn64 / (ms_f / 1e3), "ms": ms_f,
                               "hbm_frac": rn64 * 8 / (ms_f / 1e3) / 1e9 / peak, "launch": tuned64}
    rows["w64_u64"] = {"rn_s": rn64 / (ms_u / 1e3), "ms": ms_u,
                       "hbm_frac": rn64 * 8 / (ms_u / 1e3) / 1e9 / peak, "launch": tuned64u}
    one64 = Streams64(1, seeds=[W.SINGLE_STREAM["seed"]], stream=stream)
    o64 = torch.empty((1, nb), dtype=torch.int64, device="cuda")
    ms_cut64 = _time(lambda: one64.u64(nb, out=o64), stream, torch)
    one64.set_split(1)
    ms_serial64 = _time(lambda: one64.u64(nb, out=o64), stream, torch)
    one64.close()
    rows["w64_single_stream_2p20_u64"] = {"ms": ms_cut64, "rn_s": nb / (ms_cut64 / 1e3),
                                          "ms_one_warp_uncut": ms_serial64}
    ms_j = _time(lambda: s64.jump(J), stream, torch)
    rows["w64_jump_16384_streams"] = {"words": J, "set_bits": bin(J).count("1"), "ms": ms_j,
                                      "us_per_stream_application": ms_j * 1e3 / (STREAMS * bin(J).count("1"))}
    s64.close()
    del b64
    return rows


def batched_row(torch, L, stream, peak, reps=3):
    """4096 streams, one item each, lengths log-uniform in [2^10, 2^24],
    types uniform over u32/uniform/normal: one persistent-kernel launch per
    repetition (graph replay).  Also the longest item alone, which bounds the
    launch from below (one stream is a serial chain)."""
    from paper_1108_0486_gb300 import Streams
    items = W.batched_uneven()
    seeds = W.seeds(len(items))
    total = sum(it.count for it in items)
    outs = [torch.empty(it.count, dtype=torch.int32 if it.kind == 0 else torch.float32, device="cuda")
            for it in items]
    st = Streams(len(items), seeds=seeds, stream=stream)
    spec = [(it.stream, it.kind, it.count, o.data_ptr()) for it, o in zip(items, outs)]
    arr = L.make_items(spec)  # built once, outside the timed region
    # the batch kernel's shape per output type, tuned on this batch (the
    # streams are restored, so they do not advance)
    tuned = L.xg_autotune_batch(st.ctx, arr)
    shapes = {name: tuned[k][:2] for k, name in enumerate(W.KIND_NAMES)}
    # two warm-up calls: calls alternate between two launchers (so that one
    # can be planned while the other runs), and each sizes its buffers once
    ms = _time(lambda: L.xg_generate_batch(st.ctx, arr), stream, torch, reps=reps, warm=2)
    # host time of the call itself (planning and enqueueing; the GPU is idle
    # for the part of it before the first kernel is enqueued)
    host = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.xg_generate_batch(st.ctx, arr)
        host.append((time.perf_counter() - t0) * 1e3)
    torch.cuda.synchronize()
    by_piece = {}
    for q in (18, 19, 20):
        st.set_batch_split(1 << q)
        by_piece[f"2^{q}"] = _time(lambda: L.xg_generate_batch(st.ctx, arr), stream, torch, reps=reps, warm=2)
    st.set_batch_split(0)
    # the same lengths with a single output type: the batch machinery
    # against the HBM floor when no normal transform limits it
    by_type = {}
    for k, name in ((0, "u32"), (1, "uniform"), (2, "normal")):
        arr_k = L.make_items([(s_, k, c_, p_) for s_, _, c_, p_ in spec])
        ms_k = _time(lambda: L.xg_generate_batch(st.ctx, arr_k), stream, torch, reps=reps, warm=2)
        words_k = sum(it.count + (it.count & 1 if k == 2 else 0) for it in items)
        by_type[name] = {"ms": ms_k, "rn_s": total / (ms_k / 1e3),
                         "hbm_frac": total * 4 / (ms_k / 1e3) / 1e9 / peak, "words": words_k,
                         "shape": shapes[name]}
        if k < 2:
            # every shape, for the record (the tuned one is restored after)
            per_shape = {}
            for tpg, wpl in ((32, 2), (16, 4), (8, 4)):
                L.xg_set_batch_shape(st.ctx, k, tpg, wpl)
                per_shape[f"({tpg},{wpl})"] = _time(lambda: L.xg_generate_batch(st.ctx, arr_k), stream, torch,
                                                    reps=reps, warm=2)
            L.xg_set_batch_shape(st.ctx, k, *shapes[name])
            by_type[name]["ms_by_shape"] = per_shape
    longest = max(range(len(items)), key=lambda i: items[i].count)
    one = L.make_items([spec[longest]])
    ms_long = _time(lambda: L.xg_generate_batch(st.ctx, one), stream, torch, reps=reps, warm=2)
    st.close()
    del outs
    torch.cuda.empty_cache()
    return {"workload": "4096 items (streams 0..4095, seeds 1..4096), lengths log-uniform [2^10, 2^24] "
                        "(PCG64 seed 1108), types uniform over u32/uniform/normal, one graph-replayed launch",
            "rns_total": total, "ms": ms, "rn_s": total / (ms / 1e3), "host_call_ms": min(host),
            "shapes": shapes, "autotune_ms": {name: tuned[k][2] for k, name in enumerate(W.KIND_NAMES)},
            "ms_by_forced_piece_len": by_piece, "same_lengths_one_type": by_type,
            "hbm_frac": total * 4 / (ms / 1e3) / 1e9 / peak,
            "longest_item": items[longest].count, "longest_item_alone_ms": ms_long,
            "hbm_floor_ms": total * 4 / peak / 1e6}


def serving_row(torch, L, stream, seconds=10.0, plain_seconds=2.0, rate=20000.0, lanes=48, split=0,
                plain=True):
    """Open-loop Poisson arrivals at `rate` req/s on 65536 resident streams,
    sizes log-uniform in [2^10, 2^22], 60/30/10 normal/uniform/u32, memory
    cap 16 GiB (library pool).  Latency = completion (server clock,
    CLOCK_MONOTONIC) minus the request's scheduled arrival, so a submitter
    that falls behind shows up as latency; the time from submission is
    reported beside it.  Then the plain path: one xg_generate_* kernel launch
    per request (long calls not cut) on one CUDA stream, the same arrivals
    over `plain_seconds`, latency from the scheduled arrival to the request's
    CUDA event."""
    import threading as th
    from paper_1108_0486_gb300 import Streams
    S = 65536
    reqs = W.serving_requests(n_streams=S, rate=rate, duration=seconds)
    st = Streams(S, seeds=W.seeds(S), stream=stream)
    torch.cuda.synchronize()
    if split:
        st.set_batch_split(split)
    L.xg_server_start(st.ctx, 16 << 30, 1024, lanes)
    done_times = []
    refused = [0]
    n_total = len(reqs)
    cbuf = (L.XgCompletion * 4096)()

    def reaper():
        # bulk drain: one call returns (and releases) every finished request
        while len(done_times) < n_total:
            got = L.xg_collect(st.ctx, release=True, buf=cbuf)
            for tk, ts, tl, td, status, _ in got:
                done_times.append((tk, ts, tl, td))
            if not got:
                time.sleep(0.0002)

    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    rt = th.Thread(target=reaper)
    rt.start()
    t0_ns = time.monotonic_ns()
    t0 = time.perf_counter()
    for r in reqs:
        gap = r.t_arrival - (time.perf_counter() - t0)
        if gap > 3e-4:
            time.sleep(gap - 2e-4)  # release the GIL to the reaper
        while time.perf_counter() - t0 < r.t_arrival:
            pass
        while True:
            try:
                L.xg_submit(st.ctx, r.stream, r.kind, r.count, 0)
                break
            except L.XGError as e:
                if e.status != L.XG_EAGAIN:
                    raise
                refused[0] += 1
                time.sleep(0.0001)
    rt.join()
    sys.setswitchinterval(old_switch)
    wall = time.perf_counter() - t0
    stats = L.xg_server_stats_get(st.ctx)
    L.xg_server_stop(st.ctx)
    # completions come back in completion order; ticket numbers grow in
    # submission order, which is arrival order (one submitting thread)
    done_times.sort(key=lambda x: x[0])
    assert len(done_times) == len(reqs)
    arrival_ns = np.array([t0_ns + r.t_arrival * 1e9 for r in reqs])
    lat = np.array([(d - a) / 1e6 for (_, _, _, d), a in zip(done_times, arrival_ns)])
    lat_sub = np.array([(d - s) / 1e6 for _, s, _, d in done_times])
    qwait = np.array([(l - s) / 1e6 for _, s, l, _ in done_times])
    words = sum(r.count for r in reqs)
    span = (max(d for _, _, _, d in done_times) - t0_ns) / 1e9
    row = {"workload": f"65536 streams, Poisson {rate:.0f} req/s for {seconds:g} s, sizes log-uniform "
                       "[2^10, 2^22], 60/30/10 normal/uniform/u32 (PCG64 seed 486), cap 16 GiB",
           "requests": len(reqs), "rns": words, "rn_s": words / span, "offered_rn_s": words / seconds,
           "latency_from": "scheduled arrival",
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "max_ms": float(lat.max()),
           "p50_from_submit_ms": float(np.percentile(lat_sub, 50)),
           "p99_from_submit_ms": float(np.percentile(lat_sub, 99)),
           "p50_queue_ms": float(np.percentile(qwait, 50)),
           "p99_queue_ms": float(np.percentile(qwait, 99)), "refused_retries": refused[0],
           "batches": stats["batches"], "mean_batch": stats["items_launched"] / max(1, stats["batches"]),
           "server_thread_launch_busy": stats["host_launch_ns"] / 1e9 / wall, "wall_s": wall,
           "lanes": lanes, "piece_words": split or "auto"}
    if not plain:
        st.close()
        return row
    buf = torch.empty(1 << 22, dtype=torch.int32, device="cuda")
    fns = [L.xg_generate_u32, L.xg_generate_uniform, L.xg_generate_normal]

    def plain_arm(window):
        # one xg_generate_* call per request, in arrival order, on one CUDA
        # stream; latency from the scheduled arrival to the request's event
        preqs = [r for r in reqs if r.t_arrival < window]
        evs = []
        e0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        t0 = time.perf_counter()
        for r in preqs:
            while time.perf_counter() - t0 < r.t_arrival:
                pass
            fns[r.kind](st.ctx, r.stream, 1, r.count, buf.data_ptr(), r.count)
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            evs.append(e)
        torch.cuda.synchronize()
        plat = np.array([e0.elapsed_time(e) / 1e3 - r.t_arrival for e, r in zip(evs, preqs)]) * 1e3
        return {"requests": len(preqs), "window_s": window, "latency_from": "scheduled arrival",
                "p50_ms": float(np.percentile(plat, 50)), "p99_ms": float(np.percentile(plat, 99)),
                "max_ms": float(plat.max()), "drain_s": float(e0.elapsed_time(evs[-1]) / 1e3)}

    st.set_batch_split(1)
    row["plain_one_launch_per_request"] = dict(
        plain_arm(plain_seconds), kernel_launches_per_request=1,
        note="same arrivals; each request is one single-stream kernel launch (one warp), and one CUDA "
             "stream serialises them, so the queue grows")
    st.set_batch_split(0)
    row["plain_cut_by_jump_ahead"] = dict(
        plain_arm(min(plain_seconds, 0.5)),
        note="context: the same per-request calls with long calls cut into jump-ahead pieces "
             "(several launches per long request)")
    st.close()
    return row


def serving_bulk(torch, L, stream, rate, seconds, lanes=48, max_batch=1024, split=0, cap_gib=16, size_scale=1,
                 mix=(0.1, 0.3, 0.6)):
    """Open-loop Poisson arrivals at `rate`, the serving row's mix (or `mix`
    = (u32, uniform, normal) weights), submitted by one host thread in bulk
    (xg_submit_many: every request that has arrived by the time of the
    call), library pool outputs released by a reaper that drains completions
    in bulk.  Latency = completion minus arrival, both on CLOCK_MONOTONIC
    (the server's clock)."""
    import threading as th
    from paper_1108_0486_gb300 import Streams
    S = 65536
    reqs = W.serving_requests(n_streams=S, rate=rate, duration=seconds, lo=(1 << 10) * size_scale,
                              hi=(1 << 22) * size_scale, mix=mix)
    n = len(reqs)
    rec = L.make_requests([(r.stream, r.kind, r.count, 0) for r in reqs])
    arrival = np.array([r.t_arrival for r in reqs])
    tickets = np.zeros(n, dtype=np.uint64)
    st = Streams(S, seeds=W.seeds(S), stream=stream)
    torch.cuda.synchronize()
    if split:
        st.set_batch_split(split)
    L.xg_server_start(st.ctx, cap_gib << 30, max_batch, lanes)
    done = np.zeros(n, dtype=np.uint64)          # completion time per ticket order
    tick_done = np.zeros(n, dtype=np.uint64)
    got = [0]
    buf = np.zeros(65536, dtype=L.COMPLETION_DTYPE)

    collect_s = [0.0]

    def reaper():
        while got[0] < n:
            c0 = time.perf_counter()
            k = L.xg_collect_into(st.ctx, buf, release=True)
            collect_s[0] += time.perf_counter() - c0
            if k:
                tick_done[got[0]:got[0] + k] = buf["ticket"][:k]
                done[got[0]:got[0] + k] = buf["t_done_ns"][:k]
                got[0] += k
            else:
                time.sleep(0.0001)

    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    rt = th.Thread(target=reaper)
    rt.start()
    refused = 0
    calls = 0
    submit_s = 0.0
    t0 = time.monotonic_ns()
    i = 0
    while i < n:
        now = (time.monotonic_ns() - t0) / 1e9
        j = int(np.searchsorted(arrival, now, side="right"))
        if j > i:
            c0 = time.perf_counter()
            acc = L.xg_submit_many(st.ctx, rec, i, j - i, tickets)
            submit_s += time.perf_counter() - c0
            calls += 1
            if acc < j - i:
                refused += 1
                time.sleep(0.0001)
            i += acc
        else:
            time.sleep(max(0.0, min(1e-4, arrival[i] - now)))
    rt.join()
    sys.setswitchinterval(old_switch)
    wall = (time.monotonic_ns() - t0) / 1e9
    stats = L.xg_server_stats_get(st.ctx)
    L.xg_server_stop(st.ctx)
    st.close()
    # ticket numbers grow in submission order: each completion's request
    # index is its ticket's rank
    order = np.searchsorted(tickets, tick_done)
    assert np.array_equal(tickets[order], tick_done)
    t_done = np.empty(n, dtype=np.float64)
    t_done[order] = done.astype(np.float64)
    lat_ms = (t_done - (t0 + arrival * 1e9)) / 1e6
    words = int(rec["count"].sum())
    span = (t_done.max() - t0) / 1e9
    return {"offered_req_s": rate, "window_s": seconds, "requests": n,
            "submit_calls": calls, "mean_requests_per_call": n / max(1, calls),
            "delivered_rn_s": words / span, "offered_rn_s": words / seconds,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "max_ms": float(lat_ms.max()), "mean_batch": stats["items_launched"] / max(1, stats["batches"]),
            "server_thread_launch_busy": stats["host_launch_ns"] / 1e9 / wall,
            "submit_calls_busy": submit_s / wall, "collect_calls_busy": collect_s[0] / wall,
            "refused_calls": refused, "wall_s": wall}


def serving_sweep(torch, L, stream, rates=(40000.0, 160000.0, 640000.0, 1280000.0, 2560000.0), seconds=0.25):
    """Saturation sweep of the serving workload with bulk submission:
    latency (from arrival) and delivered RN/s as the Poisson rate grows past
    what the GPU can serve."""
    return [serving_bulk(torch, L, stream, rate, seconds) for rate in rates]


def serving_sweep_words(torch, L, stream, peak, rates=(320000.0, 640000.0, 1280000.0), seconds=0.25):
    """The served path without normals: the same server and bulk submission,
    requests half u32 and half uniforms of 2^12..2^24 words (log-uniform), as
    the rate passes the HBM write bound; hbm_frac = delivered bytes / the
    measured copy rate."""
    out = []
    for rate in rates:
        r = serving_bulk(torch, L, stream, rate, seconds, size_scale=4, mix=(0.5, 0.5, 0.0))
        r["hbm_frac"] = r["delivered_rn_s"] * 4 / (peak * 1e9)
        out.append(r)
    return {"workload": "65536 streams, Poisson arrivals, sizes log-uniform [2^12, 2^24], 50/50 u32/uniform "
                        "(PCG64 seed 486), cap 16 GiB, bulk submission, 0.25 s windows", "points": out}


def curand_row(torch, stream, n=1 << 30):
    """Context only: NVIDIA's XORWOW generator (the CURAND row of the paper's
    Table 1) timed through the cuRAND host API on the same GPU, 2^30 u32 and
    2^30 FP32 normals.  A library call with no parity claim."""
    import ctypes
    import glob
    paths = sorted(glob.glob("/usr/local/cuda/lib64/libcurand.so*") +
                   glob.glob("/usr/local/cuda/targets/*/lib/libcurand.so*"))
    if not paths:
        return {"unavailable": "libcurand not found"}
    lib = ctypes.CDLL(paths[0])
    gen = ctypes.c_void_p()
    if lib.curandCreateGenerator(ctypes.byref(gen), 101):  # CURAND_RNG_PSEUDO_XORWOW
        return {"unavailable": "curandCreateGenerator failed"}
    lib.curandSetStream(gen, ctypes.c_void_p(stream.cuda_stream))
    lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(1108))
    buf = torch.empty(n, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    ms_u = _time(lambda: lib.curandGenerate(gen, p, ctypes.c_size_t(n)), stream, torch)
    ms_n = _time(lambda: lib.curandGenerateNormal(gen, p, ctypes.c_size_t(n), ctypes.c_float(0.0),
                                                  ctypes.c_float(1.0)), stream, torch)
    lib.curandDestroyGenerator(gen)
    del buf
    return {"generator": "cuRAND XORWOW (library, context only)", "u32_rn_s": n / (ms_u / 1e3),
            "normal_rn_s": n / (ms_n / 1e3), "u32_ms": ms_u, "normal_ms": ms_n}


def end_to_end(st, stream, torch, L, args, dist=None, ws=1):
    """The same step through the C ABI into pinned host memory: each call
    generates on the device in pieces and copies them to the host while the
    next piece is generated; the timed region includes every copy.  With
    N ranks the job's time is the slowest rank's and the bytes are the job's."""
    host = torch.empty((STREAMS, N_PER), dtype=torch.int32, pin_memory=True)
    hostf = torch.empty((STREAMS, N_PER), dtype=torch.float32, pin_memory=True)
    ptr_u, ptr_f = host.data_ptr(), hostf.data_ptr()

    def step():
        L.xg_generate_u32(st.ctx, 0, STREAMS, N_PER, ptr_u, N_PER)
        L.xg_generate_uniform(st.ctx, 0, STREAMS, N_PER, ptr_f, N_PER)

    step()
    torch.cuda.synchronize()
    k = max(1, min(args.steps, 10))
    if dist:
        dist.barrier()
    # each call returns once its outputs are in host memory, so a step's
    # time is its wall time; the figure is the whole timed region's
    per_step = []
    t0 = time.perf_counter()
    for _ in range(k):
        ts = time.perf_counter()
        step()
        per_step.append(time.perf_counter() - ts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt * 1e3, dist, "cuda") / 1e3
    rns = STREAMS * N_PER * 2 * k * ws / dt
    # the box's own device-to-host rate into the same pinned buffer (a plain
    # 4 GiB copy, best of three), the ceiling of this end-to-end figure
    src = torch.empty((STREAMS, N_PER), dtype=torch.int32, device="cuda")
    best = None
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        best = t if best is None else min(best, t)
    del src
    box_gbs = STREAMS * N_PER * 4 / best / 1e9
    e2e_gbs = STREAMS * N_PER * 8 * k / dt / 1e9 if ws == 1 else None
    med_gbs = STREAMS * N_PER * 8 / statistics.median(per_step) / 1e9
    return {"value": rns, "unit": UNIT, "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": STREAMS * N_PER * 8 * ws, "steps": k,
            "d2h_gbs": e2e_gbs, "median_step_d2h_gbs": med_gbs, "box_d2h_copy_gbs": box_gbs,
            "frac_of_box_d2h": (e2e_gbs / box_gbs) if e2e_gbs else None,
            "note": "host buffers are pinned; no inputs cross per step (state resident); "
                    "box_d2h_copy_gbs = a plain 4 GiB device-to-host copy into the same buffer (best "
                    "of 3); single calls on this shared host are sometimes several times slower "
                    "than the rest, which the median step shows beside the whole-region figure"}


def profile_kernel(args):
    """One kernel's workload alone, for ncu captures (prints a JSON line
    marked as a profiling case; not a bench line).  --n-per sets the words
    per stream (16384 streams), or the batch's length cap."""
    import torch
    from paper_1108_0486_gb300 import Streams, _lib as L
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n = args.n_per or N_PER
    out = {"profiling_case": args.kernel, "n_per": n}
    if args.kernel in ("normal", "normal_sum", "u32", "uniform"):
        st = Streams(STREAMS, seeds=W.seeds(STREAMS), stream=stream)
        kind = "normal" if args.kernel.startswith("normal") else args.kernel
        if args.launch:
            tpg, wpl = (int(v) for v in args.launch.split(","))
            st.set_launch(kind, tpg, wpl)
            out["launch"] = {"tpg": tpg, "wpl": wpl, "block": "default of the configuration"}
        elif not args.no_autotune:
            out["launch"] = st.autotune(kind, n)
        if args.kernel == "normal_sum":
            sums = torch.empty(STREAMS, dtype=torch.float32, device="cuda")
            fn = lambda: st.normal_sum(n, out=sums)
        else:
            buf = torch.empty((STREAMS, n), dtype=torch.int32 if kind == "u32" else torch.float32,
                              device="cuda")
            fn = lambda: st.generate(kind, n, out=buf)
        out["ms"] = _time(fn, stream, torch, reps=args.steps, warm=args.warmup)
    elif args.kernel == "w64_uniform":
        from paper_1108_0486_gb300 import Streams64
        st = Streams64(STREAMS, seeds=W.seeds(STREAMS), stream=stream)
        if args.launch:
            v = [int(x) for x in args.launch.split(",")]
            block = v[2] if len(v) > 2 else 0
            st.set_launch("uniform", v[0], v[1], block)
            out["launch"] = {"tpg": v[0], "wpl": v[1], "block": block or "default of the configuration"}
        elif not args.no_autotune:
            out["launch"] = st.autotune("uniform", n)
        buf = torch.empty((STREAMS, n), dtype=torch.float64, device="cuda")
        out["ms"] = _time(lambda: st.uniform(n, out=buf), stream, torch, reps=args.steps, warm=args.warmup)
    elif args.kernel == "jump":
        # one matrix application per stream per call (2^20 has one set bit)
        st = Streams(STREAMS, seeds=W.seeds(STREAMS), stream=stream)
        out["ms"] = _time(lambda: st.jump(1 << 20), stream, torch, reps=args.steps, warm=args.warmup)
    elif args.kernel == "jump8":
        # the bench row's jump: 2^40 + 2^20 + 12345 words, 8 set bits
        st = Streams(STREAMS, seeds=W.seeds(STREAMS), stream=stream)
        J = (1 << 40) + (1 << 20) + 12345
        out["ms"] = _time(lambda: st.jump(J), stream, torch, reps=args.steps, warm=args.warmup)
    elif args.kernel == "batch":
        items = [it for it in W.batched_uneven() if it.count <= n] if args.n_per else W.batched_uneven()
        st = Streams(4096, seeds=W.seeds(4096), stream=stream)
        outs = [torch.empty(it.count, dtype=torch.int32, device="cuda") for it in items]
        arr = L.make_items([(it.stream, it.kind, it.count, o.data_ptr()) for it, o in zip(items, outs)])
        out["items"] = len(items)
        out["ms"] = _time(lambda: L.xg_generate_batch(st.ctx, arr), stream, torch, reps=args.steps,
                          warm=args.warmup)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the extra rows")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="arrival window of the serving row (10 s: about 200K requests)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default=None, choices=["u32", "uniform", "normal", "normal_sum", "batch", "w64_uniform", "jump", "jump8"],
                    help="time one kernel's workload alone (profiling case; not a bench line)")
    ap.add_argument("--n-per", type=int, default=None,
                    help="override words per stream (profiling of a smaller case; not a bench line)")
    ap.add_argument("--launch", default=None,
                    help="profiling case: fixed lanes,words per lane[,block] (e.g. 8,4) instead of autotuning "
                         "(the block applies to the 64-bit case)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured")
    ap.add_argument("--rank-check", action="store_true",
                    help="check the N-rank launcher on CPU (gloo, no GPU work; not a bench line)")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU, as a scaling run needs; the ranks re-enter here
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]))
    if args.rank_check:
        rank_check(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.n_per:
        global N_PER
        N_PER = args.n_per
        CONFIG["n_per_stream"] = N_PER
        CONFIG["workload"] = f"PROFILING CASE: {STREAMS} streams x {N_PER} words (not the bench workload)"
    if args.kernel:
        profile_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
