"""Benchmark of the V-family generation path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Workload (default): V-MT19937-32 with 16 lanes, 65536 independent generators
seeded from splitmix64(1); one step produces 2^30 uint32 followed by 2^30
float32 (24-bit conversion) from the running streams, i.e. 16384 + 16384
outputs per generator, fused into one launch.  The generators are created and
de-phased (seed + jump-ahead) before the timed region; their states stay
resident in HBM.  Every step writes 8 GiB, far more than the 129 MB L2, so no
flush is needed between steps.

The JSON line reports random GB/s written (output bytes / device time), the
HBM roofline of the generation kernel (algorithmic bytes = output + one read
and one write of every combined state), the end-to-end rate through the C ABI
into pinned host memory, the one-time initialisation cost and the oracle on
the host cores.  Under torchrun every rank runs the full per-GPU workload with
its own seeds (weak scaling); the max time over ranks is reported.
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

from paper_2309_16682_gb300 import inputs as I  # noqa: E402

METRIC = "random GB/s written (bit-exact)"
UNIT = "GB/s"
KERNELS = {"mt32": "gen_mt_kernel", "mt64": "gen_mt_kernel", "sfmt": "gen_sfmt_kernel"}
ESIZE = {"u32": 4, "f32": 4, "u64": 8, "f64": 8}


def profiled_traffic(key: str):
    """DRAM bytes per launch of a kernel from profiles/traffic.json (an ncu
    capture), or None when the kernel's sources changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)[key]
        h = hashlib.sha256()
        for src in t["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest()[:16] != t["source_sha"]:
            return None
        return float(t["traffic_bytes_per_launch"])
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    from paper_2309_16682_gb300 import shard
    shard.barrier()


def max_over_ranks(world, x: float) -> float:
    from paper_2309_16682_gb300 import shard
    return shard.max_over_ranks(x)


# ---------------------------------------------------------------------------
# oracle legs (host cores)
# ---------------------------------------------------------------------------
_POOL = {}


def _oracle_pool(workload: str, pool: int = 4):
    """Lane states of the first `pool` generators of the workload (oracle)."""
    import oracle as O
    if workload not in _POOL:
        w = I.WORKLOADS[workload]
        v = O.VARIANTS[w["variant"]]
        seeds = I.workload_seeds(workload)
        t0 = time.perf_counter()
        lanes = [O.lane_states(v, w["lanes"], int(seeds[g])) for g in range(pool)]
        _POOL[workload] = (lanes, time.perf_counter() - t0, pool)
    return _POOL[workload]


def oracle_sample(workload: str, min_seconds: float, max_gens: int = 1 << 20):
    """Time the oracle producing whole per-generator step outputs (all segments,
    interleave and conversion) until min_seconds have passed.  The lane states
    come from a small pool prepared before timing; generation cost does not
    depend on which state is used.  Returns (bytes, seconds, generators)."""
    import oracle as O
    w = I.WORKLOADS[workload]
    v = O.VARIANTS[w["variant"]]
    count = w["generators"]
    segs = [(n // count, dt) for dt, n in w["outputs"]]
    words = sum(n * O.words_per_output(v, dt) for n, dt in segs)
    lanes, _, pool = _oracle_pool(workload)
    t0 = time.perf_counter()
    nbytes, gens = 0, 0
    while gens < max_gens:
        ws = O.vstream_words(v, w["lanes"], 0, words, 0, lanes=lanes[gens % pool])
        off = 0
        for n, dt in segs:
            k = n * O.words_per_output(v, dt)
            nbytes += O.convert(v, ws[off:off + k], dt).nbytes
            off += k
        gens += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    return nbytes, time.perf_counter() - t0, gens


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(workload, seconds, steps, barrier, q):
    """One host process of the all-cores oracle timing: prepare untimed, then
    for every step meet the others at the barrier and produce for `seconds`."""
    try:
        import oracle as O
        O.prepare_all()
        _oracle_pool(workload)
        oracle_sample(workload, 0.0, max_gens=1)
        for k in range(steps):
            barrier.wait(timeout=300)
            b, t, gens = oracle_sample(workload, seconds)
            q.put((k, b, t, gens))
    except Exception as e:  # reported to the parent
        q.put((-1, "error", repr(e), 0))


def oracle_sample_procs(workload: str, seconds: float, procs: int, steps: int = 1):
    """oracle_sample in `procs` host processes at once (spawned, so safe after
    GPU work), `steps` times; returns [(bytes, seconds of the slowest,
    generators)] per step."""
    import multiprocessing as mp
    import oracle as O
    O.prepare_all()                       # polynomial caches written before the workers read them
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(workload, seconds, steps, barrier, q)) for _ in range(procs)]
    for p in ps:
        p.start()
    res = [q.get(timeout=600) for _ in range(procs * steps)]
    for p in ps:
        p.join(timeout=60)
    bad = [r for r in res if r[0] < 0]
    if bad:
        raise RuntimeError(f"oracle worker failed: {bad[0][2]}")
    out = []
    for k in range(steps):
        rk = [r for r in res if r[0] == k]
        out.append((sum(r[1] for r in rk), max(r[2] for r in rk), sum(r[3] for r in rk)))
    return out


def workload_config(workload: str, count: int, world: int, reduced: bool = False) -> dict:
    """The `config` of a bench line: the same keys for both arms."""
    w = I.WORKLOADS[workload]
    segs = [(n // w["generators"], dt) for dt, n in w["outputs"]]
    out_bytes = sum(n * count * ESIZE[dt] for n, dt in segs)
    return {"workload": workload if not reduced else f"{workload}[:{count}]",
            "variant": w["variant"], "lanes": w["lanes"],
            "generators_per_gpu": count, "outputs_per_step": [[dt, n * count] for n, dt in segs],
            "l2": "no flush: each step writes %.1f GiB (> 129 MB L2)" % (out_bytes / 2**30),
            "parallelism": f"{world} independent GPU(s), generators sharded, no collective"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle as O
    O.prepare_all()
    w = I.WORKLOADS[args.workload]
    _oracle_pool(args.workload)
    for _ in range(args.warmup):
        oracle_sample(args.workload, 0.0, max_gens=1)
    cores = host_cores()
    tot_b, tot_t, tot_g = 0, 0.0, 0
    for b, t, gens in oracle_sample_procs(args.workload, args.ref_seconds / max(args.steps, 1), cores, args.steps):
        tot_b += b
        tot_t += t
        tot_g += gens
    val = tot_b / tot_t / 1e9
    sample = (f"{tot_g} whole per-generator step outputs ({tot_b} bytes) of the {w['generators']}-generator "
              f"workload over {args.steps} steps on {cores} host processes; lane states from a pool of 4 "
              f"generators prepared untimed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": workload_config(args.workload, w["generators"], 1),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# served mix: Poisson arrivals, the continuous-batching server against the
# plain form (each request initialised and generated on its own, in arrival
# order, one after another)
# ---------------------------------------------------------------------------
NAMES = {0: "mt32", 1: "mt64", 2: "sfmt"}


def _pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def _ms(x, q):
    v = _pct(x, q)
    return None if v is None else 1e3 * v


SMALL_N = 10_000        # "small" requests: at most this many outputs


def run_served(vmt, requests: int, rate: float, plain_requests: int, client: str = "batched"):
    import torch
    tr = I.request_trace(requests, rate_per_s=rate)
    native = {0: "u32", 1: "u64", 2: "u32"}
    reqs = [(NAMES[int(tr["variant"][i])], int(tr["lanes"][i]), native[int(tr["variant"][i])],
             int(tr["seed"][i]), int(tr["jump"][i]), int(tr["n"][i]), float(tr["arrival_s"][i]))
            for i in range(requests)]
    esize = {"u32": 4, "u64": 8}
    srv = vmt.Server(state_budget=16 << 30, output_budget=96 << 30, max_batch=4096, reserve=True)
    # warm-up: polynomial tables of every variant and digit tables
    for v in ("mt32", "mt64", "sfmt"):
        rid = srv.submit(v, 4, native[{"mt32": 0, "mt64": 1, "sfmt": 2}[v]], 1, 12345, 1000)
        srv.wait(rid)
        srv.release(rid)
    torch.cuda.synchronize()
    warm_stats = srv.stats()
    # one client thread: submit the requests whose arrival time has passed,
    # and between arrivals take finished requests from the completion queue
    # (with their server-stamped latency) and release them -- in batched
    # calls, one per group, or (client="single") one call per request
    arr_t = np.array([r[6] for r in reqs])
    lag = np.zeros(requests)
    lat = np.zeros(requests)
    t0 = time.perf_counter()
    i, done, t_end = 0, 0, t0
    if client == "batched":
        carr = vmt.Server.requests([r[:6] for r in reqs])
        idx_of = {}
        while done < requests:
            now = time.perf_counter() - t0
            j = int(np.searchsorted(arr_t, now, side="right"))
            if j > i:
                ids = srv.submit_many(carr, i, j - i)
                lag[i:j] = np.maximum(0.0, time.perf_counter() - t0 - arr_t[i:j])   # submitted this late
                idx_of.update(zip(ids.tolist(), range(i, j)))
                i = j
            wait_us = int(1e6 * (arr_t[i] - now)) if i < requests else 20000
            ids, st, lt = srv.next_done_many(max(0, min(wait_us, 20000)), 4096)
            if len(ids):
                idx = np.fromiter((idx_of.pop(r) for r in ids.tolist()), np.int64, len(ids))
                lat[idx] = lt + lag[idx]
                srv.release_many(ids)
                done += len(ids)
                t_end = time.perf_counter()
    else:
        idx_of = {}
        while done < requests:
            now = time.perf_counter() - t0
            while i < requests and reqs[i][6] <= now:
                v, m, dt, seed, jump, n, arr = reqs[i]
                rid = srv.submit(v, m, dt, seed, jump, n)
                lag[i] = max(0.0, time.perf_counter() - t0 - arr)
                idx_of[rid] = i
                i += 1
            wait_us = int(1e6 * (reqs[i][6] - now)) if i < requests else 20000
            rid = srv.next_done(max(0, min(wait_us, 20000)))
            while rid is not None:
                k = idx_of.pop(rid)
                lat[k] = srv.poll(rid)[3] + lag[k]
                srv.release(rid)
                done += 1
                t_end = time.perf_counter()
                rid = srv.next_done(0)
    lat_n = [r[5] for r in reqs]
    lag_all = lag.tolist()
    lat = lat.tolist()
    stats = srv.stats()
    stats0 = warm_stats
    srv.close()
    total_bytes = sum(n * esize[dt] for (_, _, dt, _, _, n, _) in reqs)
    small = [t for t, n in zip(lat, lat_n) if n <= SMALL_N]
    batched = {"p50_ms": _ms(lat, 50), "p99_ms": _ms(lat, 99),
               "small_n_p50_ms": _ms(small, 50), "small_n_requests": len(small),
               "throughput_GBps": total_bytes / (t_end - t0) / 1e9, "batches": stats["batches"],
               "peak_output_bytes": stats["peak_output_bytes"], "wall_s": t_end - t0,
               "host_launch_s": stats["host_launch_s"] - stats0["host_launch_s"],
               "init_gpu_s": stats["init_gpu_s"] - stats0["init_gpu_s"],
               "batch_gpu_s": stats["batch_gpu_s"] - stats0["batch_gpu_s"],
               "express": {"batches": stats["express_batches"] - stats0["express_batches"],
                           "requests": stats["express_completed"] - stats0["express_completed"]},
               "mean_queued_ms": 1e3 * (stats["queued_s"] - stats0["queued_s"] + stats["express_queued_s"] -
                                        stats0["express_queued_s"]) / max(1, requests),
               "mean_running_ms": 1e3 * (stats["running_s"] - stats0["running_s"] + stats["express_running_s"] -
                                         stats0["express_running_s"]) / max(1, requests),
               "express_mean_queued_ms": 1e3 * (stats["express_queued_s"] - stats0["express_queued_s"]) /
               max(1, stats["express_completed"] - stats0["express_completed"]),
               "express_mean_running_ms": 1e3 * (stats["express_running_s"] - stats0["express_running_s"]) /
               max(1, stats["express_completed"] - stats0["express_completed"]),
               "express_gpu_span_ms_per_batch": 1e3 * (stats["express_batch_gpu_s"] - stats0["express_batch_gpu_s"]) /
               max(1, stats["express_batches"] - stats0["express_batches"]),
               "mean_submit_lag_ms": 1e3 * float(np.mean(lag_all)) if lag_all else None,
               "hw_work_queues": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
               "client": client}
    # plain form on the first plain_requests requests of the same trace
    pr = reqs[:plain_requests]
    plat, psmall = [], []
    pbytes = 0
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for (v, m, dt, seed, jump, n, arr) in pr:
        while time.perf_counter() - t0 < arr:
            pass
        g = vmt.VGenerator(v, m, [seed], [jump])
        out = g.generate(n, dt)
        stream.synchronize()
        plat.append(time.perf_counter() - t0 - arr)
        if n <= SMALL_N:
            psmall.append(plat[-1])
        pbytes += n * esize[dt]
        g.close()
        del out
    p_wall = time.perf_counter() - t0
    plain = {"p50_ms": _ms(plat, 50), "p99_ms": _ms(plat, 99), "throughput_GBps": pbytes / p_wall / 1e9,
             "small_n_p50_ms": _ms(psmall, 50), "small_n_requests": len(psmall),
             "requests": len(pr), "wall_s": p_wall}
    return {"requests": requests, "arrival_rate_per_s": rate, "lanes": "4/8/16", "length_words": "log-uniform 1e3..1e8",
            "batched": batched, "plain": plain,
            "note": "latency = the trace's arrival time to completion (server-stamped), outputs released in completion "
                    "order by a single client thread; plain = one request at a time, "
                    "vmt_init + vmt_generate + synchronise, on a prefix of the same trace; small_n = requests "
                    "of at most 10^4 outputs"}


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------


def kernel_key(workload: str) -> str:
    w = I.WORKLOADS[workload]
    return KERNELS[w["variant"]] + f"<{w['variant']}, M={w['lanes']}>"


class Generation:
    """One generation workload made resident on the GPU: its generators
    (seeded and de-phased before any timing), its output buffers and the step
    (one fused generate launch of all its output segments)."""

    def __init__(self, vmt, workload: str, seeds, count: int):
        import torch
        self.vmt, self.workload = vmt, workload
        w = I.WORKLOADS[workload]
        self.w, self.count = w, count
        self.segs = [(n // w["generators"], dt) for dt, n in w["outputs"]]   # outputs per generator
        self.out_bytes = sum(n * count * ESIZE[dt] for n, dt in self.segs)
        vmt.prepare(w["variant"])            # the variant's polynomial tables, untimed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.g = vmt.VGenerator(w["variant"], w["lanes"], seeds)
        torch.cuda.synchronize()
        self.init_s = time.perf_counter() - t0
        from paper_2309_16682_gb300 import UNITS
        unit_bytes = {"mt32": 4, "mt64": 8, "sfmt": 16}[w["variant"]]
        self.state_bytes = count * w["lanes"] * UNITS[vmt.VARIANTS[w["variant"]]] * unit_bytes
        self.outs = [torch.empty((count, n), dtype=vmt._torch_dtype(dt), device="cuda") for n, dt in self.segs]

    def step(self):
        self.g.generate_multi(self.segs, outs=self.outs)

    def autotune(self, reps: int = 3):
        """Time every compiled kernel configuration of this workload's
        (variant, lanes) on its own generator count and output mix, keep the
        fastest; returns the grid searched with each point's time."""
        v, m = self.w["variant"], self.w["lanes"]
        cands = self.vmt.tune_kernels(v, m)
        if len(cands) < 2:
            return None
        best, times = self.vmt.autotune_grid(v, m, self.count, self.segs, reps=reps)
        return {"best": best, "grid": [dict(c, ms=t) for c, t in zip(cands, times)],
                "note": "each point: mean of %d calls of the workload's step after a warm-up, better of two "
                        "alternating rounds; the timed steps use the best" % reps}

    def time_steps(self, steps: int, warmup: int, world: int, clk=None):
        """Warm-up, then `steps` timed steps between CUDA events on the
        launching stream; returns (total ms over ranks, per-step ms)."""
        import torch
        stream = torch.cuda.current_stream()
        for _ in range(max(warmup, 3)):
            self.step()
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        if clk is not None:
            clk.start()
            time.sleep(0.3)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for k in range(steps):
            self.step()
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop() if clk is not None else None
        barrier(world)
        per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
        total_ms = max_over_ranks(world, evs[0].elapsed_time(evs[-1]))
        return total_ms, per_step, clocks

    def roofline(self, launch_ms: float, peak: float, peak_kind: str, write_peak: float):
        alg = self.out_bytes + 2 * self.state_bytes
        achieved = alg / (launch_ms / 1e3) / 1e9
        out_gbs = self.out_bytes / (launch_ms / 1e3) / 1e9
        t = profiled_traffic(kernel_key(self.workload))
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "write_peak": write_peak, "frac_of_write_peak": achieved / write_peak,
                "traffic": t * self.count / self.w["generators"] if t is not None else None,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg,
                "output_only_frac": out_gbs / peak, "output_only_frac_of_write_peak": out_gbs / write_peak,
                "kernel": kernel_key(self.workload)}

    def close(self):
        self.g.close()
        self.outs = None


def run_extra_config(vmt, workload: str, steps: int, warmup: int, world: int, rank: int, peak, peak_kind,
                     write_peak, tune: bool = True):
    """The other generation workloads, timed the same way as the headline
    (every rank runs its own slice of the workload's generators)."""
    from paper_2309_16682_gb300 import shard
    w = I.WORKLOADS[workload]
    count = w["generators"]
    seeds = shard.rank_seeds(workload, world, rank, count)
    job = Generation(vmt, workload, seeds, count)
    tuned = job.autotune() if tune else None
    total_ms, per_step, _ = job.time_steps(steps, warmup, world)
    launch_ms = float(np.mean(per_step))
    res = {"workload": workload, "variant": w["variant"], "lanes": w["lanes"], "generators_per_gpu": count,
           "outputs_per_step": [[dt, n * count] for n, dt in job.segs], "steps": steps,
           "ms_per_step": total_ms / steps, "value": job.out_bytes * steps * world / (total_ms / 1e3) / 1e9,
           "unit": UNIT,
           "words_per_s": sum(n * count for n, _ in job.segs) * steps * world / (total_ms / 1e3),
           "step_ms": {"best": float(np.min(per_step)), "median": float(np.median(per_step))},
           "init_s": job.init_s, "tuning": tuned}
    if count > 1:
        res["roofline"] = job.roofline(launch_ms, peak, peak_kind, write_peak)
        if job.out_bytes < (1 << 30):
            res["l2"] = "outputs smaller than L2 stay partly cached"
    else:
        # one generator: a latency figure (one CTA does the whole call)
        res["latency_us"] = 1e3 * float(np.median(per_step))
        res["note"] = "one V-generator per call: latency-bound (a single CTA), not an HBM figure"
    job.close()
    return res


def run_gb300(args, world, rank, local):
    import torch
    import paper_2309_16682_gb300 as vmt
    w = I.WORKLOADS[args.workload]
    count = args.generators or w["generators"]
    # rank r owns generators [r * count, (r + 1) * count) of the workload's
    # global generator sequence (weak scaling, no collective on the data path)
    from paper_2309_16682_gb300 import shard
    seeds = shard.rank_seeds(args.workload, world, rank, count)
    stream = torch.cuda.current_stream()

    # one-time initialisation: seeding + jump-ahead de-phasing (timed
    # separately, after the variant's polynomial tables are built)
    job = Generation(vmt, args.workload, seeds, count)
    g, segs, outs, out_bytes = job.g, job.segs, job.outs, job.out_bytes
    init_s = job.init_s
    # the autotuner times every compiled kernel configuration on this
    # workload: its generator count and its fused output mix (both change
    # which configuration wins)
    if args.kernel >= 0:
        vmt.tune_set_kernel(w["variant"], w["lanes"], args.kernel)   # a fixed configuration (profiling)
    tuned = None if (args.no_tune or args.kernel >= 0) else job.autotune()
    if tuned is not None and args.save_tune:
        vmt.tune_save(vmt.tune_cache_path())   # kept per GPU model; vmt.tune_load reapplies it
    tune_kernel = vmt.tune_kernels(w["variant"], w["lanes"])[vmt.tune_get_kernel(w["variant"], w["lanes"])] \
        if w["variant"] != "sfmt" else None

    # the HBM write ceiling of this GPU (store-only kernel), untimed
    write_peak = vmt.measure_store_bw(8 << 30, 5)
    clk = ClockSampler(local)
    total_ms, per_step, clocks = job.time_steps(args.steps, args.warmup, world, clk)
    value = out_bytes * args.steps * world / (total_ms / 1e3) / 1e9
    # the step is one kernel launch: its average duration is the step time
    launch_ms = float(np.mean(per_step))
    peak, peak_kind = peaks()
    roof = job.roofline(launch_ms, peak, peak_kind, write_peak)

    # end to end through the C ABI into pinned host memory
    e2e = None
    if not args.no_e2e:
        hosts = [torch.empty((count, n), dtype=vmt._torch_dtype(dt), pin_memory=True) for n, dt in segs]
        for hb, (n, dt) in zip(hosts, segs):   # warm-up
            g.generate_host(n, dt, out=hb)
        barrier(world)
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            for hb, (n, dt) in zip(hosts, segs):
                g.generate_host(n, dt, out=hb)
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
        # the bound: a plain device-to-host copy of the same bytes into the same
        # pinned buffers, timed right after (the host's memory is shared with
        # other jobs, so this ceiling moves from run to run)
        copy_gbs = 0.0
        for _ in range(3):   # best of three: the host's memory is shared with other jobs
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for hb, ob in zip(hosts, outs):
                hb.copy_(ob, non_blocking=True)
            torch.cuda.synchronize()
            copy_gbs = max(copy_gbs, out_bytes / (time.perf_counter() - t1) / 1e9)
        e2e_val = out_bytes * e2e_steps * world / e2e_s / 1e9
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": out_bytes, "steps": e2e_steps,
               "d2h_copy_gbs": copy_gbs, "frac_of_d2h_copy": e2e_val / world / copy_gbs,
               "note": "vmt_generate_host into pinned host memory; the step has no host inputs (the generator "
                       "states stay resident on the GPU between calls), so nothing is copied host to device"}
        del hosts

    # jump evaluation (a3) at full size: every lane of every generator by one
    # full-degree polynomial x^d mod mu, d a 64-bit offset
    jump = None
    if not args.no_jump:
        d = int(I.splitmix64(7, 1)[0])
        jp = vmt.jump_poly(w["variant"], d)
        poly = np.zeros(312, np.uint64)          # degree < 19968 for every variant
        poly[:min(312, jp.size)] = jp[:312]
        nbits = 312 * 64
        g.jump(poly, nbits)                 # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record(stream)
        for _ in range(reps):
            g.jump(poly, nbits)
        e1.record(stream)
        torch.cuda.synchronize()
        jt = e0.elapsed_time(e1) / 1e3 / reps
        pop = int(sum(bin(int(x)).count("1") for x in poly))
        # 32-bit XOR-words per lane-jump: set coefficients x lane-state words
        lane_words = {"mt32": 624, "mt64": 624, "sfmt": 624}[w["variant"]]
        xw = count * w["lanes"] * pop * lane_words / jt
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        alu_peak = sms * 64 * sm_mhz * 1e6
        jump = {"lane_jumps": count * w["lanes"], "seconds": jt, "lane_jumps_per_s": count * w["lanes"] / jt,
                "poly_popcount": pop, "xor_words_per_s": xw, "alu_peak_lop3_per_s": alu_peak,
                "frac": xw / alu_peak, "bound": "alu",
                "note": "vmt_jump of every lane by x^d mod mu (d a 64-bit offset); 32-bit XOR-words = set "
                        "coefficients x 624 words per lane-state; peak = SMs x 64 LOP3 lanes/clk x SM clock; "
                        "a three-input XOR covers two set coefficients, so frac can exceed the pipe's share"}

    # exact single-stream mode: 2^30 outputs of ONE base generator of the
    # workload's variant (its own scalar stream), in parallel chunks
    single = None
    if not args.no_stream:
        native = {"mt32": "u32", "mt64": "u64", "sfmt": "u32"}[w["variant"]]
        ns = 1 << 30 if native == "u32" else 1 << 29
        sbuf = torch.empty(ns, dtype=vmt._torch_dtype(native), device="cuda")
        vmt.stream_generate(w["variant"], 5489, ns, native, out=sbuf)   # warm-up (polynomials cached)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            vmt.stream_generate(w["variant"], 5489, ns, native, out=sbuf)
        e1.record(stream)
        torch.cuda.synchronize()
        st_s = e0.elapsed_time(e1) / 1e3 / reps
        single = {"value": ns * sbuf.element_size() / st_s / 1e9, "unit": UNIT, "outputs": ns, "dtype": native,
                  "seconds": st_s, "note": "vmt_stream_generate: one base generator (seed 5489) cut into "
                                           "jump-started chunks; includes seeding, the chunk jumps and the "
                                           "generation"}
        del sbuf

    # buffered scalar queries on the host: one 16-lane MT32 generator, single
    # queries served from pinned buffers refilled in bulk by the GPU
    scalar = None
    if not args.no_scalar:
        sq = vmt.ScalarGenerator("mt32", 16, 5489, 0, "u32", buffer_outputs=1 << 22)
        sq.drain(1 << 24)                   # warm-up
        nq = 1 << 28
        t0 = time.perf_counter()
        sq.drain(nq)
        sq_s = time.perf_counter() - t0
        sq.close()
        scalar = {"value": nq / sq_s, "unit": "queries/s", "queries": nq, "seconds": sq_s,
                  "ms_per_1e4_queries": 1e3 * SMALL_N * sq_s / nq,
                  "note": "vmt_scalar_drain: one u32 per query from a 16-lane MT32 V-generator, buffers of 2^22 "
                          "outputs refilled by the GPU while the host reads the other one"}

    # the other generation workloads (MT19937-64 and SFMT19937 at full size,
    # and the single 4-lane generator), timed like the headline
    configs = None
    if not args.no_configs:
        g.close()
        job.close()
        outs = None
        torch.cuda.empty_cache()
        configs = {}
        for name in [n for n in I.WORKLOADS if n != args.workload]:
            configs[name] = run_extra_config(vmt, name, args.config_steps, args.warmup, world, rank, peak,
                                             peak_kind, write_peak, tune=not args.no_tune)
            torch.cuda.empty_cache()

    served = None
    if not args.no_serve:
        served = run_served(vmt, args.serve_requests, 2.0e4, args.plain_requests, args.served_client)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O
        O.prepare_all()
        _, t_pool, pool = _oracle_pool(args.workload)
        cores = host_cores()
        b, t, gens = oracle_sample_procs(args.workload, 0.6 * args.ref_seconds, cores)[0]
        b1, t1, g1 = oracle_sample(args.workload, 0.4 * args.ref_seconds)
        cpu = {"value": b / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "single_core_value": b1 / t1 / 1e9,
               "sample": f"{gens} whole per-generator step outputs ({b} bytes) in {t:.1f} s on {cores} host "
                         f"processes, and {g1} in one process in {t1:.1f} s; seed+jump of {pool} generators took "
                         f"{t_pool:.1f} s (untimed)"}

    if rank == 0:
        lane_jumps = count * w["lanes"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(args.workload, count, world, args.generators),
            "roofline": roof,
            "words_per_s": sum(n * count for n, _ in segs) * args.steps * world / (total_ms / 1e3),
            "step_ms": {"best": float(np.min(per_step)), "median": float(np.median(per_step)),
                        "mean": float(np.mean(per_step)), "each": [round(float(t), 4) for t in per_step]},
            "gpu_launches": args.steps,
            "tuning": {"kernel": tune_kernel, "autotune": tuned},
            "e2e": e2e,
            "configs": configs,
            "cpu_baseline": cpu,
            "init": {"seconds": init_s, "lane_jumps": lane_jumps, "lane_jumps_per_s": lane_jumps / init_s,
                     "note": "seed + jump-ahead de-phasing of all generators before the timed region (the "
                             "variant's polynomial tables prepared first, untimed)"},
            "jump": jump,
            "single_stream": single,
            "scalar_queries": scalar,
            "clocks": clocks,
            "served": served,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="vmt32_m16_g65536", choices=sorted(I.WORKLOADS))
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (time the table's current choice)")
    ap.add_argument("--save-tune", action="store_true", help="keep the autotuner's table in the per-GPU cache file")
    ap.add_argument("--kernel", type=int, default=-1,
                    help="time this kernel configuration index of the workload (no autotuner; for profiling)")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-mix measurement")
    ap.add_argument("--no-jump", action="store_true", help="skip the full-size jump measurement")
    ap.add_argument("--no-stream", action="store_true", help="skip the single-stream measurement")
    ap.add_argument("--no-scalar", action="store_true", help="skip the scalar-query measurement")
    ap.add_argument("--serve-requests", type=int, default=100000)
    ap.add_argument("--served-client", default="batched", choices=["batched", "single"],
                    help="the served-mix client: batched calls, or one call per request")
    ap.add_argument("--plain-requests", type=int, default=1000)
    ap.add_argument("--generators", type=int, default=0,
                    help="smaller generator count (profiling cases); default: the workload's")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other generation workloads")
    ap.add_argument("--config-steps", type=int, default=10, help="timed steps of each other generation workload")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        # host-only: no process group; under torchrun rank 0 alone runs it
        from paper_2309_16682_gb300 import shard
        world, rank, _ = shard.env_world()
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup(args.gpus)
    run_gb300(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
