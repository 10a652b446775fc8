"""Benchmark: G list elements ranked per second on a random list of n = 2^28.

One step = one lr_rank call over a uniformly random-order single list of
2^28 elements (unweighted, int32 ranks) already resident in HBM: every kernel
of the path runs (prep, head selection, chase at every level, base case,
propagation).  The inputs (1 GiB succ, 2 GiB records, 1 GiB ranks) are far
larger than L2, so no flush is needed between steps.

Printed as one JSON line (rank 0).  Extra keys:
  roofline     the level-0 chase kernel against measured HBM bandwidth, with
               64 algorithmic bytes per element (one 32 B sector gathered and
               one written back);
  pipeline     the whole step against the random-sector roofline
               (measured HBM GB/s / 64 B per element);
  cpu_baseline the CPU oracle, single thread, on a bounded sample;
  e2e          the same metric through the host-buffer pipeline
               (lr_pipeline_*: pinned host buffers, every step's copies
               inside the timed region, overlapped with the rankings).

--impl reference times the CPU oracle as the reference arm.  Under torchrun
(N > 1) every rank ranks its own list (replicas, no collective on the data
path); value is the total over ranks divided by the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G list elements ranked/s at n=2^28 (1 GB300) and % of random-sector HBM roofline"
UNIT = "G elem/s"
BYTES_PER_ELEM_CHASE = 64          # exchange form: one 32 B sector read + one 32 B sector write-back
BYTES_PER_ELEM_CHASE_LOG = 36      # log form: one 32 B sector gathered + one 4 B log entry written
# the level-0 chase kernel of each form: name, source file and the section of it
# the kernel is built from (with the device header), committed traffic record
CHASE0 = {
    "exchange": ("k_chase<Rec8> (level-0 ruler chasing, exchange form)", "lr_kernels.cu",
                 "// ---------------------------------------------------------------- chase",
                 "// ---------------------------------------------------------------- finalize",
                 "chase0_traffic.json", BYTES_PER_ELEM_CHASE),
    "log": ("k_chase_log (level-0 ruler chasing, log form)", "lr_log.cu",
            "// ---------------------------------------------------------------- log writer",
            "// ---------------------------------------------------------------- propagation",
            "chase0_log_traffic.json", BYTES_PER_ELEM_CHASE_LOG),
}
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lrk = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lrk


def init_dist(backend):
    import torch.distributed as dist
    ws, rk, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def max_over_ranks(value, dist, device="cpu"):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(step, steps, warmup, dist=None, sync=None, device="cpu"):
    """W untimed steps, then exactly K steps between barriers; returns the
    slowest rank's seconds for the K steps."""
    for _ in range(warmup):
        step()
    if sync:
        sync()
    if dist is not None:
        dist.barrier()
    if sync:
        sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    if sync:
        sync()
    t1 = time.perf_counter()
    if dist is not None:
        dist.barrier()
    return max_over_ranks(t1 - t0, dist, device)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # start timing only once nvidia-smi has initialised and sampled: its
            # start-up would otherwise overlap the first timed steps
            t_end = time.time() + 3.0
            while not self.rows and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
            self.warm = len(self.rows)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import statistics
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = self.rows[getattr(self, "warm", 0):] or self.rows   # samples of the timed region
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for nm, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        else:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        out.update(self.memory_facts())
        return out

    def memory_facts(self):
        """ECC mode and memory clock: the random-access rate differs between
        boxes, and these are the settings that could explain it."""
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(self.gpu),
                                "--query-gpu=ecc.mode.current,clocks.mem,clocks.max.mem",
                                "--format=csv,noheader,nounits"],
                               capture_output=True, text=True, timeout=20)
            ecc, mem, mem_max = [x.strip() for x in r.stdout.strip().split(",")]
            return {"ecc": ecc, "mem_mhz": float(mem), "mem_max_mhz": float(mem_max)}
        except Exception:
            return {}


def kernel_source_hash(form="exchange"):
    """Hash of the source a level-0 chase kernel is built from: the device
    header and the kernel's section of its file."""
    _, fname, start, end, _, _ = CHASE0[form]
    csrc = os.path.join(ROOT, "paper_2606_09318_gb300", "csrc")
    h = hashlib.sha256()
    with open(os.path.join(csrc, "lr_device.cuh"), "rb") as fh:
        h.update(fh.read())
    with open(os.path.join(csrc, fname), "r") as fh:
        text = fh.read()
    h.update(text[text.index(start):text.index(end)].encode())
    return h.hexdigest()[:16]


def ncu_traffic(n, form="exchange"):
    """DRAM bytes per level-0 chase launch from the committed ncu summary,
    scaled to n elements, or None if the kernel changed since the capture."""
    path = os.path.join(ROOT, "profiles", CHASE0[form][4])
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("kernel_hash") != kernel_source_hash(form):
        return None
    return float(d["dram_bytes_per_elem"]) * n


def host_cpu():
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_baseline(seconds_target=15.0, lg=26):
    """The oracle as it stands, one thread, on random lists of 2^26 (a quarter
    of the headline size: the 2^28 list takes about a minute per run)."""
    import numpy as np
    import gen
    import oracle
    oracle.build()
    n = 1 << lg
    succ = gen.random_list(n, 2028)
    t_total, reps = 0.0, 0
    while t_total < seconds_target and reps < 8:
        t0 = time.perf_counter()
        r = oracle.rank(succ)
        t_total += time.perf_counter() - t0
        reps += 1
    assert r.shape[0] == n and np.int64(r.max()) == n - 1
    out = {"value": n * reps / t_total / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "random-order list n=2^%d x %d runs (%.1f s), single thread" % (lg, reps, t_total)}
    out.update(host_cpu())
    return out


def make_random_list(n, seed, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    order = torch.randperm(n, device=device, generator=g, dtype=torch.int64)
    s = torch.empty(n, dtype=torch.int64, device=device)
    s[order[:-1]] = order[1:]
    s[order[-1]] = order[-1]
    out = s.to(torch.int32)
    del s
    return out, order


def run_ours(args):
    import torch
    import paper_2606_09318_gb300 as lr
    ws, rk, lrk = dist_env()
    torch.cuda.set_device(lrk)
    dist = init_dist("nccl")
    dev = torch.device("cuda", lrk)
    n = args.n
    lr.load()
    succ, order = make_random_list(n, 1000 * 2 + rk, dev)
    rank = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        lr.rank_ex(succ, out=rank, sync=False, stream=stream)

    # warm-up then timed region (device events + host clock around K steps)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if lr.device_status(stream) != 0:
        raise RuntimeError("device reported an error during warm-up")
    lr.profile_enable(True)
    lr.profile_read(reset=True)
    launches0 = lr.kernel_launch_count()
    # one event between consecutive steps: the whole region and every step's own time
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(lrk) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        evs[0].record(stream)
        for j in range(args.steps):
            step()
            evs[j + 1].record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    ev0, ev1 = evs[0], evs[-1]
    per_step = [evs[j].elapsed_time(evs[j + 1]) for j in range(args.steps)]
    launches = lr.kernel_launch_count() - launches0
    prof = lr.profile_read(reset=True)
    lr.profile_enable(False)
    st = lr.device_status(stream)
    if st != 0:
        raise RuntimeError("device reported %s" % lr.status_string(st))
    ms_local = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms_local, dist, device=dev)

    # correctness of the timed output (properties that determine it exactly)
    r64 = rank.to(torch.int64)
    sl = succ.to(torch.int64)
    idx = torch.arange(n, device=dev)
    term = sl == idx
    ok = bool((r64[~term] == r64[sl[~term]] + 1).all()) and int(r64[term].sum()) == 0 \
        and int(r64[order[0]]) == n - 1
    del r64, sl, idx, term
    if not ok:
        raise RuntimeError("benchmark output failed the rank recurrence check")

    # end-to-end through the host-buffer pipeline (lr_pipeline_*, pinned host
    # memory): every step copies its own input up and its ranks down inside
    # the timed region; the copies of one step run under the ranking of its
    # neighbours, and the rankings run back to back
    e2e = None
    if not args.no_e2e:
        hsucc = succ.cpu().pin_memory()
        hrank = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(args.e2e_depth)]
        pipe = lr.Pipeline(n, depth=args.e2e_depth, max_lists=1)
        for j in range(args.e2e_depth):                          # warm-up every slot
            pipe.submit(hsucc, out=hrank[j])
        pipe.wait()
        e2e_steps = max(2, args.steps)

        def estep_factory():
            i = [0]

            def estep():
                pipe.submit(hsucc, out=hrank[i[0] % args.e2e_depth])
                i[0] += 1
            return estep
        t = timed_steps(estep_factory(), e2e_steps, 0, dist, pipe.wait, dev)
        ref = rank.cpu()
        if not all(torch.equal(h, ref) for h in hrank):
            raise RuntimeError("host-buffer pipeline disagrees with the device path")
        pipe.close()
        del hsucc, hrank, ref
        e2e = {"value": round(ws * n * e2e_steps / t / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n,
               "api": "lr_pipeline (depth %d, list bound 1, %d ranking stream%s), pinned host buffers"
                      % (args.e2e_depth, 2 if args.e2e_depth >= 3 else 1, "s" if args.e2e_depth >= 3 else "")}

    hbm, src = measured_peaks()
    chase_ms = prof["ms_chase0"] / max(1, prof["chase0_launches"])
    form = "log" if prof["chase0_log_launches"] == prof["chase0_launches"] > 0 else "exchange"

    # the chase is a dependent random walk: measure the GPU's random-access
    # ceiling over the chase's own footprint (succ, 4 B per element, for the
    # log form; the 8 B records for the exchange form), same memory, same run
    probe = None
    if not args.no_probe:
        buf = torch.empty((4 if form == "log" else 8) * n + 256, dtype=torch.uint8, device=dev)
        probe = lr.probe_memory(buf, stream)
        del buf
    kname, _, _, _, _, kbytes = CHASE0[form]
    achieved = kbytes * n / (chase_ms * 1e-3) / 1e9
    value = ws * n / (ms * 1e-3) / 1e9
    sector_roof = hbm / BYTES_PER_ELEM_CHASE            # G elem/s
    steps_prof = max(1, prof["calls"])
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "step_ms": {"median": round(statistics.median(per_step), 4),
                    "mean": round(statistics.fmean(per_step), 4),
                    "min": round(min(per_step), 4), "max": round(max(per_step), 4)},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic: uniformly random-order single list (torch.randperm, seeded)",
        "config": {"workload": "single random-order list, n=2^28, unweighted, int32 ranks",
                   "n": n, "chase0_form": form,
                   "l2_policy": "inputs larger than L2 (1 GiB succ + 1 GiB log, or 2 GiB records)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kname,
                     "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "peak_source": src,
                     "traffic": ncu_traffic(n, form), "algorithmic_bytes": kbytes * n,
                     "ms_per_launch": round(chase_ms, 4),
                     # the chase's own ceiling over its footprint: independent
                     # random gathers, 8 in flight per thread (log form), or
                     # dependent gathers with an atomic exchange (exchange form)
                     "random_access_ceiling": None if probe is None else {
                         "footprint_bytes": int(probe["footprint_bytes"]),
                         "indep_gather_g_per_s": round(probe["indep_gather_gsteps"], 2),
                         "dependent_gather_g_per_s": round(probe["gather_gsteps"], 2),
                         "gather_in_2mib_region_g_per_s": round(probe["region_gather_gsteps"], 2),
                         "gather_exchange_g_per_s": round(probe["gather_xchg_gsteps"], 2),
                         "copy_gbs": round(probe["copy_gbs"], 1),
                         "ceiling": "indep_gather_g_per_s" if form == "log" else "gather_exchange_g_per_s",
                         "chase_frac_of_ceiling": round(
                             n / (chase_ms * 1e-3) / 1e9 /
                             probe["indep_gather_gsteps" if form == "log" else "gather_xchg_gsteps"], 4)}},
        "pipeline": {"random_sector_roofline_gelem_s": round(sector_roof, 2),
                     "frac": round(value / ws / sector_roof, 4),
                     "phases_ms_per_step": {k[3:]: round(prof[k] / steps_prof, 4) for k in
                                            ("ms_prep", "ms_select", "ms_chase0", "ms_chase_rest",
                                             "ms_base", "ms_finalize")}},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    # the batched and served forms (configs 4 and 5) on the same GPU, one
    # replica only: the batch against the per-instance loop, the server
    # against per-request plain launches on one trace of fresh requests
    if ws == 1 and not args.no_batch:
        line["batch"] = batch_measure(5, 3, dev)
        torch.cuda.empty_cache()
    if ws == 1 and not args.no_serve:
        res, info = serve_measure(300, 30, [0.5, 0.8, 0.95, 2.0], args.serve_streams, args.serve_capacity, dev)
        line["serve"] = dict({"loads": res}, **info)
        torch.cuda.empty_cache()
    if rk == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rk == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    ws, rk, _ = dist_env()
    if rk != 0:
        return
    import numpy as np
    import gen
    import oracle
    oracle.build()
    n = 1 << 24
    succ = gen.random_list(n, 4242)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.rank(succ)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    assert int(np.int64(r.max())) == n - 1
    t = sum(times)
    value = n * len(times) / t / 1e9
    sample = "random-order list n=2^24 per step (bounded sample of the n=2^28 workload), single thread"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t / len(times), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "single random-order list, n=2^28, unweighted, int32 ranks",
                   "n": 1 << 28, "sample_n": n, "parallelism": "single GPU"},
        "cpu_baseline": dict({"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": sample}, **host_cpu()),
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference_sweep(args):
    """The oracle on the sizes and orders of the size sweep, one thread on the
    host cores: random, locality (windows of 256) and identity order at
    2^20, 2^24 and 2^28, and the random order at 2^30; unweighted, int32
    ranks.  One JSON line per case (the best of --oracle-reps runs at
    2^20 and 2^24, one run above), with the rank recurrence checked."""
    ws, rk, _ = dist_env()
    if rk != 0:
        return
    import numpy as np
    import gen
    import oracle
    oracle.build()
    cases = [(lg, kind) for lg in (int(x) for x in args.oracle_sizes.split(","))
             for kind in ("random", "locality", "identity")]
    if args.oracle_top:
        cases.append((args.oracle_top, "random"))
    for lg, kind in cases:
        n = 1 << lg
        succ = gen.list_of_order_kind(kind, n, gen.config_seed(2, lg))
        reps = args.oracle_reps if lg <= 24 else 1
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            r = oracle.rank(succ)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        s64 = succ.astype(np.int64)
        term = s64 == np.arange(n, dtype=np.int64)
        ok = bool((r[~term].astype(np.int64) == r[s64[~term]].astype(np.int64) + 1).all()) \
            and int(r[term].astype(np.int64).sum()) == 0 and int(term.sum()) == 1
        print(json.dumps({"impl": "reference", "workload": "sweep", "kind": "oracle", "cores": 1,
                          "n": n, "log2n": lg, "order": kind, "weights": "none -> int32 ranks",
                          "runs": reps, "s": round(best, 4),
                          "m_elem_s": round(n / best / 1e6, 3), "exact": ok}), flush=True)
        del succ, r, s64, term


def _device_random_order(m, g, dev):
    import torch
    return torch.randperm(m, device=dev, generator=g, dtype=torch.int64)


def _device_locality_order(m, g, dev, window=256):
    import torch
    full = (m // window) * window
    order = torch.arange(m, device=dev, dtype=torch.int64)
    if full:
        keys = torch.rand(full // window, window, device=dev, generator=g)
        idx = torch.argsort(keys, dim=1) + torch.arange(0, full, window, device=dev).unsqueeze(1)
        order[:full] = idx.reshape(-1)
    if full < m:
        order[full:] = full + torch.randperm(m - full, device=dev, generator=g)
    return order


def _fill_succ(succ_view, order):
    """succ_view[order[i]] = order[i+1] (local ids), tail points to itself."""
    succ_view[order[:-1]] = order[1:].to(succ_view.dtype)
    succ_view[order[-1]] = order[-1].to(succ_view.dtype)


def batch_measure(steps, warmup, dev, k=1024, quick=False):
    """Config 4: 1024 independent random-order instances, sizes floor(2^U),
    U ~ U[8,22], int64 weights in [0, 2^20): one CUDA-graph replay of the
    autotuned batched call per step, against a host loop of one lr_rank_ex
    call per instance.  Returns a dict; `exact` is the full recurrence over
    every instance plus equality with the per-instance loop.
    k < 1024 keeps the first k of the same instances (a smaller case for
    profiling); quick skips the autotuner and the loop (default tuning, and
    `exact` is the recurrence alone)."""
    import numpy as np
    import torch
    import gen
    import paper_2606_09318_gb300 as lr
    lens = gen.batch_lengths(1024, gen.config_seed(4), 8.0, 22.0)[:k]
    offsets = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    n = int(offsets[-1])
    g = torch.Generator(device=dev)
    g.manual_seed(4000)
    succ = torch.empty(n, dtype=torch.int32, device=dev)
    for j in range(k):
        a, b = int(offsets[j]), int(offsets[j + 1])
        _fill_succ(succ[a:b], _device_random_order(b - a, g, dev))
    w = torch.randint(0, 1 << 20, (n,), dtype=torch.int64, device=dev, generator=g)
    d_off = torch.from_numpy(offsets).to(dev)
    out_b = torch.empty(n, dtype=torch.int64, device=dev)
    out_l = None if quick else torch.empty(n, dtype=torch.int64, device=dev)
    # autotune the batched shape on this input (untimed); the batched call
    # below passes no tuning, so it takes the tuned entry from the table
    t_tune = time.perf_counter()
    tuned = None if quick else lr.autotune(succ=succ, weight=w, offsets=d_off, max_lists=k)
    t_tune = time.perf_counter() - t_tune
    ws = torch.empty(lr.workspace_size(n, k, weighted=True, max_lists=k), dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream()
    kw = dict(out=out_b, max_lists=k, n_total=n, sync=False, stream=s, workspace=ws)
    with torch.cuda.stream(s):
        lr.rank_batch(d_off, succ, w, **kw)
    s.synchronize()
    assert lr.device_status(s) == 0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        lr.rank_batch(d_off, succ, w, **kw)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    with torch.cuda.stream(s):
        ms_b = timed(graph.replay, steps, warmup)
    if quick:
        assert lr.device_status(s) == 0
        del graph, ws
        inst = torch.repeat_interleave(torch.arange(k, device=dev), torch.from_numpy(lens).to(dev))
        sg = d_off[inst] + (succ.to(torch.int64) & 0xFFFFFFFF)
        del inst
        exact = _check_recurrence(sg, w, out_b, dev, global_succ=True)
        return {"metric": "G list elements ranked/s, %d instances in one CUDA graph" % k,
                "value": round(n / (ms_b * 1e-3) / 1e9, 4), "unit": UNIT, "ms_per_step": round(ms_b, 3),
                "steps": steps, "n_total": n, "k": k, "dtype": "i64 weights, i64 ranks", "exact": exact,
                "config": {"workload": "batched: the first %d of the 1024 random-order instances, "
                                       "default tuning, graph-captured" % k}}
    with torch.cuda.stream(s):
        views = [(int(offsets[j]), int(offsets[j + 1])) for j in range(k)]

        def loop():
            for a, b in views:
                lr.rank_ex(succ[a:b], w[a:b], out=out_l[a:b], max_lists=1, sync=False, stream=s)
        launches0 = lr.kernel_launch_count()
        loop_steps = max(1, steps // 4)
        ms_l = timed(loop, loop_steps, 1)
        per_loop_launches = (lr.kernel_launch_count() - launches0) / (loop_steps + 1)
    assert lr.device_status(s) == 0
    del graph, ws
    inst = torch.repeat_interleave(torch.arange(k, device=dev), torch.from_numpy(lens).to(dev))
    sg = d_off[inst] + (succ.to(torch.int64) & 0xFFFFFFFF)
    del inst
    exact = bool(torch.equal(out_b, out_l)) and _check_recurrence(sg, w, out_b, dev, global_succ=True)
    lr.autotune_clear()
    return {"metric": "G list elements ranked/s, %d instances in one CUDA graph" % k,
            "value": round(n / (ms_b * 1e-3) / 1e9, 4), "unit": UNIT, "ms_per_step": round(ms_b, 3),
            "steps": steps, "n_total": n, "k": k, "dtype": "i64 weights, i64 ranks", "exact": exact,
            "per_instance_loop": {"value": round(n / (ms_l * 1e-3) / 1e9, 4), "ms_per_step": round(ms_l, 3),
                                  "steps": loop_steps, "kernel_launches_per_step": per_loop_launches},
            "speedup_vs_loop": round(ms_l / ms_b, 3),
            "autotuned": {"f0_inv": tuned.f0_inv, "f_inv": tuned.f_inv, "cutoff": tuned.cutoff,
                          "chase_block": tuned.chase_block, "seconds": round(t_tune, 2)},
            "config": {"workload": "batched: 1024 random-order instances, sizes floor(2^U), U~U[8,22], "
                                   "int64 weights in [0,2^20), graph-captured, autotuned"}}


def run_batch(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    d = batch_measure(args.steps, args.warmup, dev, k=args.batch_k, quick=args.batch_quick)
    d["workload"] = "batch"
    print(json.dumps(d), flush=True)


def serve_measure(requests, warmup, loads, streams, capacity, dev, fresh_bytes=100e9, lo_exp=10.0,
                  hi_exp=26.0, alone_min_n=0):
    """Config 5: a Poisson request stream, sizes floor(2^U) with U ~ U[10,26],
    random or locality order with p = 0.5, int64 weights, 40 GB budget;
    continuous batching against plain per-request launches on the same
    trace, at each offered load: a fraction of the batched capacity in
    elements/s, measured first by submitting the whole trace at once
    (capacity <= 0), or of the capacity given.  Requests are generated on
    the device before the trace, every one distinct while their arrays fit
    `fresh_bytes` (then reused round-robin).
    Returns ({load: {"batched": ..., "plain": ...}}, info)."""
    import threading as th
    import numpy as np
    import torch
    import gen
    import paper_2606_09318_gb300 as lr
    g = torch.Generator(device=dev)
    g.manual_seed(5000)
    total = requests + warmup
    _, sizes, kinds, _ = gen.serving_trace(total, gen.config_seed(5), rate_per_s=1.0, lo_exp=lo_exp,
                                           hi_exp=hi_exp)
    pool, used = [], 0
    for i in range(total):
        m = int(sizes[i])
        if used + 20 * m > fresh_bytes:
            break
        order = _device_random_order(m, g, dev) if kinds[i] == "random" else _device_locality_order(m, g, dev)
        sc = torch.empty(m, dtype=torch.int32, device=dev)
        _fill_succ(sc, order)
        del order
        pool.append((sc, torch.randint(0, 1 << 20, (m,), dtype=torch.int64, device=dev, generator=g),
                     torch.empty(m, dtype=torch.int64, device=dev)))
        used += 20 * m
    pool_n = len(pool)
    mean_n = float(np.mean(sizes[:total]))

    def run_trace(mode, gaps):
        srv = lr.Server(budget_bytes=40_000_000_000, n_streams=streams, max_batch=256,
                        plain=(mode == "plain"), alone_min_n=alone_min_n)
        tickets = [None] * total
        t_start = time.perf_counter()

        def submitter():
            t = t_start
            for i in range(total):
                t += gaps[i]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                sc, wv, ov = pool[i % pool_n]
                tickets[i] = srv.submit(sc, wv, out=ov)
        thr = th.Thread(target=submitter)
        thr.start()
        lat, elems, t_first, t_last = [], 0, None, None
        for i in range(total):
            while tickets[i] is None:
                time.sleep(0.0002)
            _, info = srv.wait(tickets[i])
            if i >= warmup:
                lat.append(info["t_done_ms"] - info["t_submit_ms"])
                elems += pool[i % pool_n][0].numel()
                t_first = info["t_submit_ms"] if t_first is None else min(t_first, info["t_submit_ms"])
                t_last = info["t_done_ms"] if t_last is None else max(t_last, info["t_done_ms"])
        thr.join()
        st = srv.stats()
        srv.close()
        lat = np.array(lat)
        # served results equal the requests ranked alone (a sample)
        exact = all(bool(torch.equal(ov, lr.rank(sc, wv))) for sc, wv, ov in pool[:min(pool_n, 16)])
        return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "g_elem_s": round(elems / ((t_last - t_first) * 1e-3) / 1e9, 4),
                "batches": int(st["batches"]), "ranked_alone": int(st["ranked_alone"]),
                "exact": exact}

    measured = None
    if capacity <= 0:
        # saturation: the whole trace submitted at once, batched
        measured = run_trace("batched", np.zeros(total))
        capacity = measured["g_elem_s"] * 1e9
    out = {}
    for load in loads:
        rate = load * capacity / mean_n
        gaps = np.random.default_rng(55).exponential(1.0 / rate, size=total)
        out[str(load)] = {mode: run_trace(mode, gaps) for mode in ("batched", "plain")}
    info = {"requests": requests, "warmup": warmup, "distinct_requests": pool_n, "mean_request": mean_n,
            "capacity_elem_s": capacity, "capacity_source": "measured" if measured else "given",
            "streams": streams, "size_exp": [lo_exp, hi_exp], "alone_min_n": alone_min_n}
    if measured:
        info["saturation"] = measured
    return out, info


def run_serve(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    loads = [float(x) for x in str(args.load).split(",")]
    res, info = serve_measure(args.requests, args.serve_warmup, loads, args.serve_streams,
                              args.serve_capacity, dev, lo_exp=args.serve_lo, hi_exp=args.serve_hi,
                              alone_min_n=args.serve_alone_min)
    top = res[str(loads[-1])]
    print(json.dumps(dict({
        "workload": "serve", "metric": "served G list elements/s and p50/p99 latency",
        "value": top["batched"]["g_elem_s"], "unit": UNIT, "loads": res,
        "config": {"workload": "serving: Poisson arrivals, sizes floor(2^U) U~U[%g,%g], random/locality "
                               "orders p=0.5, int64 weights, 40 GB budget, device-resident inputs"
                               % (args.serve_lo, args.serve_hi)}}, **info)),
          flush=True)


def _device_identity_order(m, dev):
    import torch
    return torch.arange(m, device=dev, dtype=torch.int64)


def _time_call(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _check_recurrence(succ, w, rank, dev, global_succ=False):
    """Exactness at sizes the oracle cannot reach in seconds: tail 0 and
    rank[i] = w[i] + rank[succ[i]] on every element (wrapping as int64).
    global_succ: succ already holds int64 global ids (a batch)."""
    import torch
    n = succ.numel()
    sl = succ if global_succ else succ.to(torch.int64) & 0xFFFFFFFF
    idx = torch.arange(n, device=dev)
    term = sl == idx
    r = rank.to(torch.int64)
    ww = torch.ones(n, dtype=torch.int64, device=dev) if w is None else w.to(torch.int64)
    tail_ok = bool((r[term] == 0).all())
    diff = r[~term] - ww[~term] - r[sl[~term]]
    if rank.dtype == torch.int32:               # int32 ranks wrap modulo 2^32
        diff = diff % (1 << 32)
    return tail_ok and bool((diff == 0).all())


def run_sweep(args):
    """Configurations beyond the headline, one JSON line per case: the size
    sweep 2^24..2^30 in three orders, unweighted and with int32 weights in
    [-1000, 1000] (int64 ranks); the forest of 2^27 elements; the Euler tour
    of a random recursive tree with 2^26 vertices (+-1 int32 weights, int32
    ranks).  Every output is checked with the rank recurrence."""
    import numpy as np
    import torch
    import gen
    import paper_2606_09318_gb300 as lr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    g = torch.Generator(device=dev)
    g.manual_seed(2024)
    sizes = [int(x) for x in args.sweep_sizes.split(",")]
    cases = []
    for lg in sizes:
        for kind in ("random", "locality", "identity"):
            for weighted in (False, True):
                cases.append((lg, kind, weighted))
    for lg, kind, weighted in cases:
        n = 1 << lg
        order = {"random": lambda: _device_random_order(n, g, dev),
                 "locality": lambda: _device_locality_order(n, g, dev),
                 "identity": lambda: _device_identity_order(n, dev)}[kind]()
        succ = torch.empty(n, dtype=torch.int32, device=dev)
        _fill_succ(succ, order)
        del order
        w = torch.randint(-1000, 1001, (n,), dtype=torch.int32, device=dev, generator=g) if weighted else None
        out = torch.empty(n, dtype=torch.int64 if weighted else torch.int32, device=dev)
        ms = _time_call(lambda: lr.rank_ex(succ, w, out=out, sync=False), args.steps, args.warmup)
        assert lr.device_status() == 0
        ok = _check_recurrence(succ, w, out, dev)
        print(json.dumps({"workload": "sweep", "n": n, "log2n": lg, "order": kind,
                          "weights": "int32 [-1000,1000] -> int64 ranks" if weighted else "none -> int32 ranks",
                          "ms": round(ms, 3), "g_elem_s": round(n / (ms * 1e-3) / 1e9, 3),
                          "exact": ok}), flush=True)
        del succ, w, out
        torch.cuda.empty_cache()
    # forest: 16 lists of 2^22 plus geometric(mean 64) lists, labels permuted (host generator)
    fs, nl = gen.forest(1 << 27, gen.config_seed(3), n_long=16, long_len=1 << 22, mean_short=64)
    succ = torch.from_numpy(fs.view(np.int32)).to(dev)
    out = torch.empty(succ.numel(), dtype=torch.int32, device=dev)
    ms = _time_call(lambda: lr.rank_ex(succ, out=out, sync=False), args.steps, args.warmup)
    assert lr.device_status() == 0
    print(json.dumps({"workload": "sweep", "case": "forest 2^27 (16 x 2^22 + geometric mean 64)",
                      "n": int(succ.numel()), "lists": nl, "ms": round(ms, 3),
                      "g_elem_s": round(succ.numel() / (ms * 1e-3) / 1e9, 3),
                      "exact": _check_recurrence(succ, None, out, dev)}), flush=True)
    del succ, out
    parent = gen.random_recursive_tree(1 << 26, gen.config_seed(3, 1))
    es, ew = gen.euler_tour(parent)
    del parent
    succ = torch.from_numpy(es.view(np.int32)).to(dev)
    w = torch.from_numpy(ew).to(dev)
    out = torch.empty(succ.numel(), dtype=torch.int32, device=dev)
    ms = _time_call(lambda: lr.rank_ex(succ, w, out=out, sync=False), args.steps, args.warmup)
    assert lr.device_status() == 0
    print(json.dumps({"workload": "sweep", "case": "Euler tour of a random recursive tree, 2^26 vertices",
                      "n": int(succ.numel()), "ms": round(ms, 3),
                      "g_elem_s": round(succ.numel() / (ms * 1e-3) / 1e9, 3),
                      "exact": _check_recurrence(succ, w, out, dev)}), flush=True)


def run_pd_compare(args):
    """The paper's comparison of the sparse ruling set with pointer doubling
    (Sections 1 and 3), on one GPU: random-order single lists of 2^20..2^28
    (and the locality order at 2^28), unweighted, int32 ranks, ranked by the
    default algorithm and by whole-list Wyllie pointer doubling
    (lr_tuning.algorithm = LR_ALGO_WYLLIE).  One JSON line per size; both
    outputs are checked with the rank recurrence."""
    import torch
    import paper_2606_09318_gb300 as lr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    g = torch.Generator(device=dev)
    g.manual_seed(2025)
    pd = lr.Tuning(algorithm=lr.ALGO_WYLLIE)
    hbm, src = measured_peaks()
    sizes = [int(x) for x in args.pd_sizes.split(",")]
    cases = [(lg, "random") for lg in sizes] + [(max(sizes), "locality")]
    for lg, kind in cases:
        n = 1 << lg
        order = (_device_random_order(n, g, dev) if kind == "random" else _device_locality_order(n, g, dev))
        succ = torch.empty(n, dtype=torch.int32, device=dev)
        _fill_succ(succ, order)
        del order
        out_s = torch.empty(n, dtype=torch.int32, device=dev)
        out_p = torch.empty(n, dtype=torch.int32, device=dev)
        ms_s = _time_call(lambda: lr.rank_ex(succ, out=out_s, sync=False), args.steps, args.warmup)
        assert lr.device_status() == 0
        ms_p = _time_call(lambda: lr.rank_ex(succ, out=out_p, tuning=pd, sync=False),
                          max(3, args.steps // 4), args.warmup)
        assert lr.device_status() == 0
        exact = _check_recurrence(succ, None, out_s, dev) and bool(torch.equal(out_s, out_p))
        rounds = max(1, (n - 1).bit_length())
        # a Wyllie round streams 8 B in and 8 B out per element and gathers one
        # random 32 B sector per unfinished element (at most n)
        gb_round = n * (16 + 32) / 1e9
        print(json.dumps({"workload": "pd_compare", "n": n, "log2n": lg, "order": kind,
                          "srs_ms": round(ms_s, 3), "srs_g_elem_s": round(n / (ms_s * 1e-3) / 1e9, 3),
                          "wyllie_ms": round(ms_p, 3), "wyllie_g_elem_s": round(n / (ms_p * 1e-3) / 1e9, 3),
                          "wyllie_rounds": rounds, "wyllie_ms_per_round": round(ms_p / rounds, 3),
                          "wyllie_round_gbs_bound": round(gb_round / (ms_p / rounds * 1e-3), 1),
                          "hbm_peak_gbs": hbm, "peak_source": src,
                          "srs_speedup": round(ms_p / ms_s, 2), "exact": exact}), flush=True)
        del succ, out_s, out_p
        torch.cuda.empty_cache()


def run_outputs(args):
    """The extra outputs of Section 1.1 (lr_rank_outputs: terminal ids,
    head-relative ranks, the inclusive form) against the plain rank on the
    same list: a random list and the 2^27 forest, unweighted and with int32
    weights (int64 ranks).  One JSON line per case; every output is checked
    (the rank recurrence, terminals shared along each list, prefix + rank
    equal at the terminal's total, the inclusive form = rank + the terminal's
    weight)."""
    import numpy as np
    import torch
    import gen
    import paper_2606_09318_gb300 as lr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    g = torch.Generator(device=dev)
    g.manual_seed(2626)
    n = args.n
    order = _device_random_order(n, g, dev)
    rsucc = torch.empty(n, dtype=torch.int32, device=dev)
    _fill_succ(rsucc, order)
    del order
    fs, _ = gen.forest(1 << 27, gen.config_seed(3), n_long=16, long_len=1 << 22, mean_short=64)
    fsucc = torch.from_numpy(fs.view(np.int32)).to(dev)
    del fs
    for name, succ in (("random list n=%d" % n, rsucc), ("forest 2^27", fsucc)):
        m = succ.numel()
        for weighted in (False, True):
            w = torch.randint(-1000, 1001, (m,), dtype=torch.int32, device=dev, generator=g) if weighted else None
            rdt = torch.int64 if weighted else torch.int32
            out = torch.empty(m, dtype=rdt, device=dev)
            term = torch.empty(m, dtype=torch.int32, device=dev)
            pre = torch.empty(m, dtype=rdt, device=dev)
            ms_plain = _time_call(lambda: lr.rank_ex(succ, w, out=out, sync=False), args.steps, args.warmup)
            plain = out.clone()
            ms_ext = _time_call(lambda: lr.rank_outputs(succ, w, term=term, prefix=pre, out=out, sync=False),
                                args.steps, args.warmup)
            assert lr.device_status() == 0
            sl = succ.to(torch.int64) & 0xFFFFFFFF
            tl = term.to(torch.int64) & 0xFFFFFFFF
            ok = bool(torch.equal(out, plain)) and _check_recurrence(succ, w, out, dev)
            ok = ok and bool((sl[tl] == tl).all()) and bool((tl[sl] == tl).all())
            ok = ok and bool(((pre.to(torch.int64) + out.to(torch.int64)) == pre.to(torch.int64)[tl]).all())
            incl = torch.empty_like(out)
            lr.rank_outputs(succ, w, term=False, prefix=False, inclusive_tail=True, out=incl)
            wt = torch.zeros(m, dtype=torch.int64, device=dev) if w is None else w.to(torch.int64)
            ok = ok and bool(torch.equal(incl.to(torch.int64), out.to(torch.int64) + wt[tl]))
            print(json.dumps({"workload": "outputs", "case": name, "n": m,
                              "weights": "int32 [-1000,1000] -> int64 ranks" if weighted else "none -> int32 ranks",
                              "rank_ms": round(ms_plain, 3), "outputs_ms": round(ms_ext, 3),
                              "outputs_g_elem_s": round(m / (ms_ext * 1e-3) / 1e9, 3),
                              "overhead": round(ms_ext / ms_plain, 3), "exact": ok}), flush=True)
            del w, out, term, pre, plain, incl, sl, tl, wt
            torch.cuda.empty_cache()


def run_probe_sweep(args):
    """Random-access rates of the GPU against the footprint the accesses
    cover (lr_probe_memory on buffers of 32 MiB .. 4 GiB): dependent 4-byte
    gathers (the chase's access), independent gathers with 8 in flight per
    thread, the same confined to one 2 MiB region per warp and round, and
    dependent 8-byte atomic exchanges.  One JSON line per footprint."""
    import torch
    import paper_2606_09318_gb300 as lr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    for lg in [int(x) for x in args.probe_sizes.split(",")]:
        buf = torch.empty((1 << lg) + 256, dtype=torch.uint8, device=dev)
        r = lr.probe_memory(buf)
        del buf
        torch.cuda.empty_cache()
        print(json.dumps({"workload": "probe", "footprint_mib": (1 << lg) >> 20,
                          "dependent_gather_g_per_s": round(r["gather_gsteps"], 2),
                          "indep_gather_g_per_s": round(r["indep_gather_gsteps"], 2),
                          "gather_in_2mib_region_g_per_s": round(r["region_gather_gsteps"], 2),
                          "dependent_exchange_g_per_s": round(r["gather_xchg_gsteps"], 2),
                          "copy_gbs": round(r["copy_gbs"], 1)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 28)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-probe", action="store_true", help="skip the random-access probe")
    ap.add_argument("--e2e-depth", type=int, default=3,
                    help="e2e: slots of the host-buffer pipeline (3 or more rank two lists at a time)")
    ap.add_argument("--no-batch", action="store_true", help="headline: skip the batched (config 4) object")
    ap.add_argument("--no-serve", action="store_true", help="headline: skip the serving (config 5) object")
    ap.add_argument("--pd-sizes", default="20,22,24,26,28", help="log2 sizes of --workload pd")
    ap.add_argument("--batch-k", type=int, default=1024,
                    help="batch: rank the first K of the 1024 instances (a smaller case for profiling)")
    ap.add_argument("--batch-quick", action="store_true",
                    help="batch: default tuning, no autotuner and no per-instance loop")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch", "serve", "sweep", "pd", "probe", "outputs"],
                    help="single: the headline (default); batch / serve: the batched and serving sets; "
                         "sweep: sizes and orders; pd: against whole-list pointer doubling; "
                         "probe: random-access rates against footprint; outputs: terminal ids, "
                         "head-relative and inclusive ranks against the plain rank")
    ap.add_argument("--probe-sizes", default="25,26,27,28,29,30,31,32",
                    help="probe: log2 footprints in bytes")
    ap.add_argument("--requests", type=int, default=2000, help="serve: measured requests")
    ap.add_argument("--sweep-sizes", default="24,26,28,30", help="sweep: log2 sizes")
    ap.add_argument("--oracle-sizes", default="20,24,28",
                    help="reference sweep: log2 sizes timed in all three orders")
    ap.add_argument("--oracle-top", type=int, default=30,
                    help="reference sweep: log2 size also timed in random order (0: none)")
    ap.add_argument("--oracle-reps", type=int, default=3, help="reference sweep: runs at n <= 2^24")
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--load", default="0.5,0.8,0.95,2.0",
                    help="serve: offered loads, as fractions of the capacity (comma-separated)")
    ap.add_argument("--serve-capacity", type=float, default=0.0,
                    help="serve: capacity in elements/s (0: measured first, the whole trace at once)")
    ap.add_argument("--serve-lo", type=float, default=10.0, help="serve: request sizes floor(2^U), U >= this")
    ap.add_argument("--serve-hi", type=float, default=26.0, help="serve: request sizes floor(2^U), U <= this")
    ap.add_argument("--serve-alone-min", type=int, default=0,
                    help="serve: requests of at least this many elements are ranked alone (0: default 2^20; "
                         "-1: never)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if args.workload == "sweep":
            run_reference_sweep(args)
        else:
            run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "pd":
        run_pd_compare(args)
    elif args.workload == "probe":
        run_probe_sweep(args)
    elif args.workload == "outputs":
        run_outputs(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
