"""Benchmark: the full 77,169-neuron microcircuit on one GB300.

One bench "step" = one persistent launch that simulates 1 s of biological
time (10,000 time steps of 0.1 ms) of the full microcircuit (~3e8 synapses).
The default run (warmup 3, steps 10) times 10 s of biological time, the
paper's run length, after 3 s of warm-up that absorb the initial transient.

Printed JSON line (rank 0):
  value            synaptic events / s (device-timed, CUDA events on the
                   library's stream), whole job over all ranks
  real_time_factor wall time / biological time (< 1: faster than real time)
  e2e              same metric through the public C ABI with the spike
                   raster read back to host memory every step
  roofline         the step kernel's algorithmic bytes (4 B per synaptic
                   event: one packed synaptic word) / its launch time, over
                   the measured HBM copy bandwidth
  cpu_baseline     the CPU oracle timed on a bounded sample of the same
                   workload on this host

--impl reference times the CPU oracle itself (the reference arm).
Multi-GPU (torchrun, --gpus N): N independent replicas, one per GPU.

The default line also carries, each with its own device timing, roofline and
clock record (skipped with --no-extras): deliver_20000 (the partition-word
delivery of 20,000-spike lists at scale 1), scale4 (1 s biological of the 4x
network), batch64 (1 s biological of 64 instances) and grad_config3 (one
forward + backward of the 10 % network over 200 ms).

Other workloads (--workload; the default line is the full microcircuit):
  scale4  the 4x microcircuit (308,676 neurons, ~1.2e9 synapses), same metric
  batch   64 independent microcircuits at scales U(0.05, 0.25) in one
          persistent kernel replayed from a CUDA graph; 1 step = 1 s
          biological of every instance; synaptic events/s over all instances
  grad    one surrogate-gradient evaluation (forward with checkpoints every
          100 steps + backward) of the 10 % microcircuit over 200 ms
  deliver the delivery kernels alone on spike lists of 25 / 93 / 4,000 /
          20,000 random sources at scales 1 and 4 (HBM roofline per case)
  realtime the full microcircuit paced to wall-clock time (one 0.1 ms step per
          0.1 ms) for --steps biological seconds: deadlines missed, step-end
          intervals
  soak    a long run of --steps biological seconds with the raster streamed
          to the host every second, then a resume-from-checkpoint check
"""
import argparse
import json
import os
import signal
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "real-time factor and synaptic events/s (full microcircuit, 1 GB300); % HBM roofline"
UNIT = "synaptic events/s"
STEPS_PER_BENCH_STEP = 10000          # 1 s of biological time at dt = 0.1 ms
BYTES_PER_EVENT = 4                   # one packed synaptic word read per event
TILING_NAMES = ["warp", "block", "partition", "words", "cluster", "stream"]   # snn_deliver tilings
# DRAM bytes (read + write) per synaptic event of k_step, from one ncu capture
# of the current kernel on the small case (scale 0.4: dram__bytes_read.sum +
# dram__bytes_write.sum of one 2000-step launch that delivered 19,040.77
# events per step); the full-size launch's traffic is taken as this figure
# times its events (re-measure whenever k_step changes)
K_STEP_DRAM_BYTES_PER_EVENT = (108.322560e6 + 3.360512e6) / (2000 * 19040.7745)
K_STEP_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one 2000-step "
                         "k_step launch at scale 0.4 (30,868 neurons, 192 MB of rows): 2.93 B "
                         "per synaptic event, times this launch's events; a lower estimate at "
                         "full size, where fewer rows stay L2-resident between spikes")
# k_deliver_words, 20,000-spike lists on the small case (scale 0.4): ncu
# dram__bytes_read + write of three launches over their mean synaptic events
K_DELIVER_WORDS_DRAM_BYTES_PER_EVENT = ((135.067904 + 135.324672 + 135.687424) +
                                        (3.596288 + 3.186432 + 3.619328)) * 1e6 / 3.0 / 31.06e6


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def reduce_over_ranks(total_ms, units, device):
    """Whole-job figures of N replicas: the slowest rank's time (max) and the
    units (synaptic events) of all ranks (sum).  One rank: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(units)
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])),
                "sm_max_mhz": float(max(r[1] for r in rows)), "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(cfg, n_threads_build, skip_steps, sample_steps):
    """Time the CPU oracle's step loop on a bounded sample of the workload."""
    import oracle
    t0 = time.time()
    net = oracle.Network(cfg, n_threads=n_threads_build)
    build_s = time.time() - t0
    sim = oracle.Simulation(net)
    sim.run(skip_steps)
    c0 = sim.counters()
    t1 = time.perf_counter()
    sim.run(sample_steps)
    dt = time.perf_counter() - t1
    c1 = sim.counters()
    events = c1["events"] - c0["events"]
    bio = sample_steps * cfg["dt"] * 1e-3
    return {"value": events / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "steps %d..%d of the full microcircuit (seed %d), %.3f s biological, "
                      "single-threaded step loop; network built untimed with %d threads in %.1f s"
                      % (skip_steps, skip_steps + sample_steps, cfg["seed"], bio,
                         n_threads_build, build_s),
            "real_time_factor": dt / bio, "seconds": dt}


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on this host's cores."""
    import workload
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cfg = workload.microcircuit(args.scale)
    import oracle
    nthreads = os.cpu_count() or 1
    t0 = time.time()
    net = oracle.Network(cfg, n_threads=nthreads)
    build_s = time.time() - t0
    sim = oracle.Simulation(net)
    chunk = args.ref_chunk
    for _ in range(args.warmup):
        sim.run(chunk)
    c0 = sim.counters()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        sim.run(chunk)
    dt = time.perf_counter() - t1
    c1 = sim.counters()
    events = c1["events"] - c0["events"]
    value = events / dt
    bio = args.steps * chunk * cfg["dt"] * 1e-3
    sample = ("each step %d time steps (%.1f ms biological) of the full microcircuit after "
              "%d warm-up steps; single-threaded oracle step loop; network built untimed "
              "with %d threads in %.1f s" % (chunk, chunk * cfg["dt"], args.warmup, nthreads,
                                             build_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/i32",
            "data": "synthetic", "real_time_factor": dt / bio,
            "config": {"workload": "full microcircuit, 77,169 LIF neurons, ~3e8 synapses, "
                                   "Poisson background, dt 0.1 ms",
                       "scale": args.scale, "seed": cfg["seed"],
                       "time_steps_per_step": chunk},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Other forms of the path, timed on bounded samples inside the default run so
# that each has its own device timing, roofline and clock record
# ---------------------------------------------------------------------------
def _events_timer(torch, stream):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    return a, b


def extra_deliver(pkg, workload, torch, stream, hbm_peak, peak_kind, m=20000, n_lists=16):
    """Stand-alone delivery of m-spike lists at scale 1 with the partition-word
    tiling (k_deliver_words): each timed launch gets a fresh list from a pool
    whose rows (n_lists x ~0.3 GB) exceed L2 many times."""
    net = pkg.Microcircuit(workload.microcircuit(1.0), stream=stream)
    rp, _, _ = net.export_network(rows_only=True)
    row_len = np.diff(rp.astype(np.int64))
    rng = np.random.default_rng(20000)
    lists = [np.sort(rng.choice(net.n, m, replace=False)).astype(np.int32) for _ in range(n_lists)]
    dev = [torch.from_numpy(x).cuda() for x in lists]
    events = float(np.mean([row_len[x].sum() for x in lists]))
    for k in range(3):
        net.deliver(dev[k].data_ptr(), m, k, 3)
    torch.cuda.synchronize()
    e0, e1 = _events_timer(torch, stream)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for k in range(n_lists):
            net.deliver(dev[k].data_ptr(), m, 7 + k, 3)
        e1.record(stream)
        torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / n_lists
    net.close()
    gbs = BYTES_PER_EVENT * events / (us * 1e-6) / 1e9
    return {"metric": "synaptic events/s of one %d-spike delivery (full microcircuit)" % m,
            "value": events / (us * 1e-6), "unit": UNIT, "us_per_list": us, "events_per_list": events,
            "launches": n_lists, "gpu_launches": n_lists,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak,
                         "traffic": K_DELIVER_WORDS_DRAM_BYTES_PER_EVENT * events,
                         "peak_kind": peak_kind, "kernel": "k_deliver_words"},
            "clocks": clk.summary(),
            "config": {"workload": "snn_deliver tiling 3 (partition words), %d random sources "
                                   "per list, %d lists" % (m, n_lists), "scale": 1.0}}


def extra_scale4(pkg, workload, torch, stream, hbm_peak, peak_kind):
    """The 4x microcircuit (308,676 neurons, ~1.2e9 synapses): one launch of
    1 s biological after a 0.2 s warm-up launch."""
    cfg = workload.microcircuit(4.0)
    net = pkg.Microcircuit(cfg, stream=stream)
    info = net.info()
    net.step(2000)
    net.sync()
    net.read_spikes_into(np.zeros(max(1, net.raster_size()), np.uint32),
                         np.zeros(max(1, net.raster_size()), np.uint32))
    c0 = net.counters()
    e0, e1 = _events_timer(torch, stream)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        net.step(STEPS_PER_BENCH_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c1 = net.counters()
    net.close()
    ev = c1["events"] - c0["events"]
    gbs = BYTES_PER_EVENT * ev / (ms * 1e-3) / 1e9
    return {"metric": "synaptic events/s (4x microcircuit)", "value": ev / (ms * 1e-3),
            "unit": UNIT, "real_time_factor": ms * 1e-3 / (STEPS_PER_BENCH_STEP * cfg["dt"] * 1e-3),
            "us_per_time_step": ms * 1e3 / STEPS_PER_BENCH_STEP,
            "spikes_per_time_step": (c1["spikes"] - c0["spikes"]) / STEPS_PER_BENCH_STEP,
            "gpu_launches": 1,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "k_step (persistent step kernel)"},
            "clocks": clk.summary(),
            "config": {"workload": "4x microcircuit, %d neurons, %d synapses, 1 launch of %d "
                                   "time steps (1 s biological)"
                                   % (info["n_neurons"], info["n_synapses"], STEPS_PER_BENCH_STEP),
                       "scale": 4.0, "ring_in_shared": info["ring_in_shared"],
                       "rows_gb": info["slot_bytes"] / 1e9}}


def extra_batch(pkg, workload, torch, stream, hbm_peak, peak_kind, n_inst=64):
    """64 microcircuits at scales U(0.05, 0.25) in one persistent kernel
    replayed from a CUDA graph: 1 s biological of every instance."""
    b = pkg.MicrocircuitBatch(workload.batched_instances(n_inst, seed=7), stream=stream)
    info = b.info(0)
    b.step(1000)
    b.sync()
    ev0 = sum(b.counters(k)["events"] for k in range(len(b)))
    e0, e1 = _events_timer(torch, stream)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        b.step(STEPS_PER_BENCH_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ev = sum(b.counters(k)["events"] for k in range(len(b))) - ev0
    launches = STEPS_PER_BENCH_STEP // info["graph_steps"]
    b.close()
    gbs = BYTES_PER_EVENT * ev / (ms * 1e-3) / 1e9
    return {"metric": "synaptic events/s of %d independent microcircuits in one persistent kernel"
                      % n_inst,
            "value": ev / (ms * 1e-3), "unit": UNIT,
            "real_time_factor": ms * 1e-3 / (STEPS_PER_BENCH_STEP * 1e-4),
            "us_per_time_step": ms * 1e3 / STEPS_PER_BENCH_STEP, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "k_batch (persistent batched step kernel)"},
            "clocks": clk.summary(),
            "config": {"workload": "%d instances, scales U(0.05, 0.25) (seed 7), %d neurons in "
                                   "total, %d time steps of every instance (1 s biological) as "
                                   "graph replays of %d steps"
                                   % (n_inst, info["n_neurons_total"], STEPS_PER_BENCH_STEP,
                                      info["graph_steps"])}}


def extra_grad(pkg, workload, torch, stream, reps=3):
    """One surrogate-gradient evaluation of the 10 % microcircuit over 200 ms
    (2000 steps, checkpoints every 100): forward, backward, through the
    torch.autograd.Function; wall time per evaluation (device-synchronised).
    The value is taken with checkpoints every 100 steps, the backward
    re-running each segment (trace budget 0); the same gradient, bit for bit,
    with the forward recording the whole trajectory instead is timed beside
    it."""
    from paper_1909_08665_gb300.autograd import microcircuit_rates
    cfg = workload.microcircuit(0.1)
    targets = torch.as_tensor(workload.target_rates())
    net = pkg.Microcircuit(cfg, stream=stream)
    start = net.save_state()
    n_steps, every = 2000, 100

    def one():
        scales = torch.ones(8, 8, dtype=torch.float64, requires_grad=True)
        nu = torch.tensor(float(cfg["nu_bg"]), dtype=torch.float64, requires_grad=True)
        rates = microcircuit_rates(scales, nu, net, n_steps, every, start)
        loss = ((rates - targets) ** 2).mean()
        loss.backward()
        return float(loss.item()), float(scales.grad.abs().max())

    def timed(budget):
        net.set_grad_trace_budget(budget)
        one()
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            res = one()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        return 1e3 * float(np.median(times)), res

    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, (loss, gmax) = timed(0)
        ms_rec, _ = timed(4 << 30)
    net.close()
    return {"metric": "surrogate-gradient evaluations/s (10% microcircuit, 200 ms, rate MSE)",
            "value": 1e3 / ms, "unit": "gradients/s", "ms_per_gradient": ms, "reps": reps,
            "loss": loss, "grad_abs_max": gmax,
            "note": "the adjoint grows ~e^0.039 per step through the chaotic dynamics: over "
                    "200 ms max|g| reaches ~4e31, so the gradient's value is dominated by that "
                    "growth; the figure times the computation, not its usefulness for training",
            "ms_per_gradient_recorded_trajectory": ms_rec,
            # per gradient: one k_step per checkpoint segment forward, k_step +
            # k_adjoint_part per segment backward, the fold and the reduction
            "gpu_launches": 3 * ((n_steps + every - 1) // every) + 2,
            "clocks": clk.summary(),
            "config": {"workload": "10%% microcircuit (7,717 neurons), %d time steps, checkpoints "
                                   "every %d steps, gradient w.r.t. 64 projection scales and nu"
                                   % (n_steps, every)}}


def run_ours(args):
    import torch

    import paper_1909_08665_gb300 as pkg
    import workload

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cfg = workload.microcircuit(args.scale, seed=12345 + rank)
    chunk = args.chunk
    t_build = time.time()
    net = pkg.Microcircuit(cfg, stream=stream)
    build_s = time.time() - t_build
    info = net.info()

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        net.step(chunk)
    net.sync()
    n_pending = max(1, net.raster_size())
    net.read_spikes_into(np.zeros(n_pending, np.uint32), np.zeros(n_pending, np.uint32))

    # -------- device-timed region: K launches, inputs (1.2 GB rows) > L2 --------
    c0 = net.counters()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for k in range(args.steps):
            starts[k].record(stream)
            net.step(chunk)
            ends[k].record(stream)
        t_all1.record(stream)
        barrier()
    net.sync()
    c1 = net.counters()
    total_ms = t_all0.elapsed_time(t_all1)

    # -------- one more launch, untimed, recording the device clock at the
    # end of every step (the real-time criterion) and the per-step synapse
    # counts (spikes, events, busiest partition, empty pairs) --------
    step_clock = torch.zeros(chunk, dtype=torch.int64, device=dev)
    step_counts = torch.zeros(4 * chunk, dtype=torch.int32, device=dev)
    net.record_step_times(step_clock.data_ptr(), chunk)
    net.record_step_counts(step_counts.data_ptr(), chunk)
    net.step(chunk)
    net.sync()
    net.record_step_times(None)
    net.record_step_counts(None)
    dts = np.diff(step_clock.cpu().numpy()) * 1e-3            # us
    step_times = {"mean_us": float(dts.mean()) if dts.size else None,
                  "p99_us": float(np.percentile(dts, 99)) if dts.size else None,
                  "max_us": float(dts.max()) if dts.size else None,
                  "steps_over_100us": int((dts > 100.0).sum()),
                  "source": "device clock at the end of each step (CTA 0) of one recorded "
                            "launch of %d steps after the timed region, its first step "
                            "excluded" % chunk}
    counts = step_counts.cpu().numpy().view(np.uint32).reshape(-1, 4).astype(np.int64)
    n_p = info["n_part"]
    step_counts_summary = {
        "busiest_partition_spikes": {"mean": float(counts[:, 2].mean()),
                                     "p99": float(np.percentile(counts[:, 2], 99)),
                                     "max": int(counts[:, 2].max())},
        "spikes_per_step": {"mean": float(counts[:, 0].mean()),
                            "p99": float(np.percentile(counts[:, 0], 99)),
                            "max": int(counts[:, 0].max())},
        "empty_pairs_fraction": float(counts[:, 3].sum() / max(1, n_p * counts[:, 0].sum())),
        "flushed": 0,
        "source": "snn_record_step_counts over the recorded launch: spikes a partition "
                  "processed (non-empty runs onto it), and (spike, partition) pairs with no "
                  "target there"}
    per_launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    events = c1["events"] - c0["events"]
    spikes = c1["spikes"] - c0["spikes"]
    total_ms, events_all = reduce_over_ranks(total_ms, events, dev)
    value = events_all / (total_ms * 1e-3)
    bio_s = args.steps * chunk * cfg["dt"] * 1e-3
    rtf = (total_ms * 1e-3) / bio_s

    # -------- end to end through the C ABI: raster read to host each step --------
    cap = 1 << 24
    h_steps = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    h_ids = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    net.read_spikes_into(h_steps, h_ids)
    barrier()
    e0 = net.counters()["events"]
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(args.steps):
        net.step(chunk)
        n = net.read_spikes_into(h_steps, h_ids)
        d2h += 8 * n + 8 * 3
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_events = net.counters()["events"] - e0
    e2e_value = e2e_events * ws / e2e_s

    hbm_peak, peak_kind = load_peaks()
    avg_launch_s = float(np.mean(per_launch_ms)) * 1e-3
    achieved = BYTES_PER_EVENT * (events / args.steps) / avg_launch_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/i32", "data": "synthetic",
        "real_time_factor": rtf,
        "config": {"workload": "%s, %d LIF neurons, %d synapses, Poisson background, dt 0.1 "
                               "ms; 1 step = %d time steps (%g s biological)"
                               % ("full microcircuit" if args.scale == 1.0
                                  else "%gx microcircuit%s" % (args.scale, " (same in-degrees)"
                                                               if args.scale > 1.0 else ""),
                                  info["n_neurons"], info["n_synapses"], chunk, chunk * 1e-4),
                   "scale": args.scale, "seed": cfg["seed"], "time_steps_per_step": chunk,
                   "l2": "no flush: synapse rows (%.2f GB) exceed the 129 MB L2"
                         % (info["n_synapses"] * 4 / 1e9),
                   "n_part": info["n_part"], "ring_in_shared": info["ring_in_shared"],
                   "slot_gb": info["slot_bytes"] / 1e9,
                   "parallelism": "replicas" if ws > 1 else "single"},
        "spikes_per_time_step": spikes / (args.steps * chunk),
        "events_per_time_step": events / (args.steps * chunk),
        "us_per_time_step": total_ms * 1e3 / (args.steps * chunk),
        "step_time": step_times,
        "step_counts": step_counts_summary,
        "build_s": build_s,
        "clocks": clk.summary(),
        "gpu_launches": args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h // max(args.steps, 1),
                "real_time_factor": e2e_s / bio_s},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak,
                     "traffic": (K_STEP_DRAM_BYTES_PER_EVENT * events / args.steps
                                 if args.scale == 1.0 else None),
                     "traffic_source": K_STEP_TRAFFIC_SOURCE if args.scale == 1.0 else None,
                     "peak_kind": peak_kind, "kernel": "k_step (persistent step kernel)"},
    }
    if rank == 0 and ws == 1 and not args.no_extras and args.scale == 1.0:
        net.close()
        line["deliver_20000"] = extra_deliver(pkg, workload, torch, stream, hbm_peak, peak_kind)
        line["scale4"] = extra_scale4(pkg, workload, torch, stream, hbm_peak, peak_kind)
        line["batch64"] = extra_batch(pkg, workload, torch, stream, hbm_peak, peak_kind)
        line["grad_config3"] = extra_grad(pkg, workload, torch, stream)
        line["gpu_launches_extras"] = sum(line[k]["gpu_launches"] for k in
                                          ("deliver_20000", "scale4", "batch64", "grad_config3"))
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.scale <= 1.0:
        line["cpu_baseline"] = cpu_baseline(cfg, os.cpu_count() or 1, args.cpu_skip,
                                            args.cpu_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args):
    import torch

    import paper_1909_08665_gb300 as pkg
    import workload

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cfgs = workload.batched_instances(args.instances, seed=7 + rank)
    t_build = time.time()
    b = pkg.MicrocircuitBatch(cfgs, stream=stream)
    build_s = time.time() - t_build
    info = b.info(0)
    chunk = args.chunk
    for _ in range(args.warmup):
        b.step(chunk)
    b.sync()
    for k in range(len(b)):
        b.read_spikes(k)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize(dev)

    ev0 = sum(b.counters(k)["events"] for k in range(len(b)))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            starts[k].record(stream)
            b.step(chunk)
            ends[k].record(stream)
        barrier()
    b.sync()
    ev1 = sum(b.counters(k)["events"] for k in range(len(b)))
    total_ms = starts[0].elapsed_time(ends[-1])
    events = ev1 - ev0
    total_ms, events_all = reduce_over_ranks(total_ms, events, dev)
    bio_s = args.steps * chunk * 1e-4
    launches_per_step = chunk // info["graph_steps"] + (1 if chunk % info["graph_steps"] else 0)
    avg_launch_s = total_ms * 1e-3 / (args.steps * launches_per_step)
    hbm_peak, peak_kind = load_peaks()
    achieved = BYTES_PER_EVENT * (events / (args.steps * launches_per_step)) / avg_launch_s / 1e9
    tilings = [b.info(k)["tiling"] for k in range(len(b))]
    # end to end through the C ABI: every instance's raster read to the host
    # after every bench step
    barrier()
    e0 = sum(b.counters(k)["events"] for k in range(len(b)))
    t0 = time.perf_counter()
    d2h = 0
    h_steps = torch.empty(1 << 22, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    h_ids = torch.empty(1 << 22, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    for _ in range(args.steps):
        b.step(chunk)
        for k in range(len(b)):
            d2h += 8 * b.read_spikes_into(k, h_steps, h_ids)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_events = sum(b.counters(k)["events"] for k in range(len(b))) - e0
    line = {
        "metric": METRIC, "value": events_all / (total_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/i32",
        "data": "synthetic", "real_time_factor": total_ms * 1e-3 / bio_s,
        "config": {"workload": "%d independent microcircuits, scales U(0.05, 0.25) (seed 7), "
                               "%d neurons in total, one persistent kernel per graph replay of "
                               "%d time steps; 1 step = %d time steps of every instance"
                               % (len(b), info["n_neurons_total"], info["graph_steps"], chunk),
                   "time_steps_per_step": chunk, "instances": len(b),
                   "tilings": {"warp_per_spike": tilings.count(0),
                               "block_per_row": tilings.count(1), "flat": tilings.count(2)},
                   "l2": "no flush: the instances' synapse rows (%.2f GB) exceed L2"
                         % (sum(b.info(k)["n_synapses"] for k in range(len(b))) * 4 / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "us_per_time_step": total_ms * 1e3 / (args.steps * chunk),
        "events_per_time_step": events / (args.steps * chunk),
        "build_s": build_s, "clocks": clk.summary(),
        "gpu_launches": args.steps * launches_per_step,
        "e2e": {"value": e2e_events * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h // max(args.steps, 1),
                "real_time_factor": e2e_s / bio_s},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                     "kernel": "k_batch (persistent batched step kernel)"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_deliver(args):
    """Delivery microbenchmark (a5 alone): one spike list of m random sources
    through snn_deliver, for m = 25 (mean activity), 93 (peak), 4,000 (the
    initial transient) and 20,000, at scale 1 and 4.  Each repetition draws a
    fresh list from a pool whose rows together exceed L2 several times."""
    import torch

    import paper_1909_08665_gb300 as pkg
    import workload

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    hbm_peak, peak_kind = load_peaks()
    rows = []
    rng = np.random.default_rng(99)
    scales = [float(x) for x in args.deliver_scale.split(",")]
    sizes = [int(x) for x in args.deliver_spikes.split(",")]
    tilings = [int(x) for x in args.deliver_tilings.split(",")]
    for scale in scales:
        net = pkg.Microcircuit(workload.microcircuit(scale), stream=stream)
        rp, _, _ = net.export_network(rows_only=True)
        row_len = np.diff(rp.astype(np.int64))
        for m in sizes:
            for tiling in tilings:
                # pool of lists: at least 1 GB of rows in total, 8 lists minimum
                per_list = float(row_len.mean()) * 4 * m
                n_lists = int(min(256, max(8, np.ceil(1.0e9 / per_list))))
                lists = [np.sort(rng.choice(net.n, m, replace=False)).astype(np.int32)
                         for _ in range(n_lists)]
                dev = [torch.from_numpy(x).cuda() for x in lists]
                events = [int(row_len[x].sum()) for x in lists]
                try:                                             # warm-up
                    for k in range(min(3, n_lists)):
                        net.deliver(dev[k].data_ptr(), m, k, tiling)
                except pkg.SnnError as err:
                    if err.code != pkg.SNN_ERR_UNSUPPORTED:
                        raise
                    rows.append({"scale": scale, "spikes": m,
                                 "tiling": TILING_NAMES[tiling],
                                 "unsupported": str(err)})
                    continue
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                reps = n_lists
                e0.record(stream)
                for k in range(reps):
                    net.deliver(dev[k].data_ptr(), m, 7 + k, tiling)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                ev = float(np.mean(events[:reps]))
                gbs = 4.0 * ev / (ms * 1e-3) / 1e9
                rows.append({"scale": scale, "spikes": m,
                             "tiling": TILING_NAMES[tiling],
                             "us": ms * 1e3, "events": ev, "achieved_gbs": gbs,
                             "frac": gbs / hbm_peak})
        net.close()
    best = max((r for r in rows if "achieved_gbs" in r), key=lambda r: r["achieved_gbs"])
    line = {
        "metric": "synaptic events/s of the delivery kernels alone (one spike list per launch)",
        "value": best["events"] / (best["us"] * 1e-6), "unit": "synaptic events/s", "n_gpus": 1,
        "steps": None, "warmup": 3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": {"workload": "snn_deliver of random spike lists at scales 1 and 4; lists drawn "
                               "from pools of >= 1 GB of rows (no list repeats within a timing)"},
        "roofline": {"bound": "hbm", "achieved": best["achieved_gbs"], "peak": hbm_peak,
                     "unit": "GB/s", "frac": best["frac"],
                     "traffic": (K_DELIVER_WORDS_DRAM_BYTES_PER_EVENT * best["events"]
                                 if best["tiling"] == "words" and best["scale"] == 1.0
                                 and best["spikes"] == 20000 else None),
                     "peak_kind": peak_kind, "kernel": "k_deliver_%s" % best["tiling"]},
        "cases": rows,
    }
    print(json.dumps(line), flush=True)


def run_realtime(args):
    """True real time (Sec. 4.1): the full microcircuit paced at one 0.1 ms
    step per 0.1 ms of wall time (snn_set_realtime) for --steps seconds of
    biological time in one launch, the raster read to the host afterwards.
    Reports the wall time per biological second, the deadlines missed (a step
    ending more than 0.1 ms after its release) and the intervals between step
    ends on the device clock."""
    import torch

    import paper_1909_08665_gb300 as pkg
    import workload

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cfg = workload.microcircuit(args.scale, seed=12345)
    period_ns = int(round(cfg["dt"] * 1e6))           # dt in ms
    n = args.steps * STEPS_PER_BENCH_STEP
    # the whole paced run is one launch: room on the device for all its spikes
    # (2^28 entries, split evenly over the partitions)
    net = pkg.Microcircuit(cfg, stream=stream, raster_capacity=1 << 28)
    for _ in range(args.warmup):                       # unpaced
        net.step(STEPS_PER_BENCH_STEP)
    net.sync()
    pending = max(1, net.raster_size())
    net.read_spikes_into(np.zeros(pending, np.uint32), np.zeros(pending, np.uint32))
    clock = torch.zeros(n, dtype=torch.int64, device="cuda")
    net.record_step_times(clock.data_ptr(), n)
    net.set_realtime(period_ns)
    c0 = net.counters()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        net.step(n)
        net.sync()
        wall = time.perf_counter() - t0
    rt = net.realtime_stats()
    net.set_realtime(0)
    net.record_step_times(None)
    c1 = net.counters()
    steps_host, ids_host = net.read_spikes()
    d_us = np.diff(clock.cpu().numpy()) * 1e-3
    bio_s = n * cfg["dt"] * 1e-3
    net_name = ("full microcircuit" if args.scale == 1.0
                else "%gx microcircuit (same in-degrees)" % args.scale)
    line = {
        "metric": "wall-clock seconds per biological second, paced at one 0.1 ms step per "
                  "0.1 ms (true real time, %s, 1 GB300)" % net_name,
        "value": wall / bio_s, "unit": "s/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/i32",
        "data": "synthetic",
        "config": {"workload": "%s paced to wall-clock time, %d time steps "
                               "(%g s biological) in one launch" % (net_name, n, bio_s),
                   "scale": args.scale, "period_ns": period_ns,
                   "l2": "no flush: synapse rows exceed L2"},
        "deadlines_missed": rt["missed"], "max_lateness_us": rt["max_late_ns"] * 1e-3,
        "step_end_interval_us": {"median": float(np.median(d_us)), "p01": float(np.percentile(d_us, 1)),
                                 "p99": float(np.percentile(d_us, 99)), "max": float(d_us.max())},
        "spikes": int(c1["spikes"] - c0["spikes"]), "spikes_read": int(steps_host.size),
        "events": int(c1["events"] - c0["events"]),
        "clocks": clk.summary(),
        "gpu_launches": 1,
    }
    print(json.dumps(line), flush=True)


def run_soak(args):
    """Long run (the paper reports several 12 h simulations, Sec. 5): the full
    microcircuit for --steps biological seconds, one second per launch, the
    raster streamed to pinned host memory after every second and checked
    against the device's spike count.  Then a resume check: the state saved at
    the end, one more second simulated, and the same second simulated again by
    a second network instance that loaded the saved state; the two rasters
    must be identical."""
    import torch

    import paper_1909_08665_gb300 as pkg
    import workload

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cfg = workload.microcircuit(args.scale, seed=12345)
    chunk = STEPS_PER_BENCH_STEP
    net = pkg.Microcircuit(cfg, stream=stream)
    bounds = np.cumsum([0] + list(cfg["pop_sizes"]))
    sizes = np.asarray(cfg["pop_sizes"], np.float64)
    cap = 1 << 24
    h_steps = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    h_ids = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    counts = np.zeros((args.steps, len(sizes)), np.int64)
    drained = 0
    c0 = net.counters()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            net.step(chunk)
            m = net.read_spikes_into(h_steps, h_ids)
            drained += m
            pops = np.searchsorted(bounds, h_ids[:m], side="right") - 1
            counts[k] = np.bincount(pops, minlength=len(sizes))[:len(sizes)]
        wall = time.perf_counter() - t0
    c1 = net.counters()
    rates = counts / sizes[None, :] / (chunk * cfg["dt"] * 1e-3)
    # resume from a saved state in a second instance of the network
    snap = net.save_state()
    net.step(chunk)
    a = net.read_spikes()
    other = pkg.Microcircuit(cfg, stream=stream)
    other.load_state(snap)
    other.step(chunk)
    b = other.read_spikes()
    resume_ok = bool(a[0].size > 0 and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]))
    other.close()
    net.close()
    bio_s = args.steps * chunk * cfg["dt"] * 1e-3
    line = {
        "metric": "wall-clock seconds per biological second of a long run, raster streamed to "
                  "the host every biological second (full microcircuit, 1 GB300)",
        "value": wall / bio_s, "unit": "s/s", "n_gpus": 1, "steps": args.steps, "warmup": 0,
        "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/i32", "data": "synthetic",
        "config": {"workload": "full microcircuit, %g s biological, 1 s per launch, raster "
                               "drained to pinned host memory after every launch" % bio_s,
                   "scale": args.scale},
        "spikes_counted": int(c1["spikes"] - c0["spikes"]), "spikes_drained": int(drained),
        "events": int(c1["events"] - c0["events"]),
        "rate_hz_mean": [float(x) for x in rates.mean(axis=0)],
        "total_rate_hz_per_second": {"min": float((counts.sum(1) / sizes.sum()).min()),
                                     "max": float((counts.sum(1) / sizes.sum()).max())},
        "resume_bit_identical": resume_ok,
        "clocks": clk.summary(),
        "gpu_launches": args.steps + 2,
        "e2e": {"value": wall / bio_s, "unit": "s/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 8 * drained // max(args.steps, 1)},
    }
    print(json.dumps(line), flush=True)


def run_grad(args):
    import torch

    import paper_1909_08665_gb300 as pkg
    from paper_1909_08665_gb300.autograd import microcircuit_rates
    import workload

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cfg = workload.microcircuit(0.1, seed=12345 + rank)
    targets = torch.as_tensor(workload.target_rates())
    net = pkg.Microcircuit(cfg, stream=stream)
    start = net.save_state()
    n_steps, every = 2000, 100
    # 0: checkpoints every 100 steps, the backward re-running each segment;
    # larger: the forward records the whole trajectory when it fits
    net.set_grad_trace_budget(args.grad_trace_budget)
    recorded = 5 * n_steps * net.n <= args.grad_trace_budget

    def one():
        scales = torch.ones(8, 8, dtype=torch.float64, requires_grad=True)
        nu = torch.tensor(float(cfg["nu_bg"]), dtype=torch.float64, requires_grad=True)
        rates = microcircuit_rates(scales, nu, net, n_steps, every, start)
        loss = ((rates - targets) ** 2).mean()
        loss.backward()
        return loss.item(), scales.grad, nu.grad

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize(dev)
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            loss, gs, gn = one()
            times.append(time.perf_counter() - t0)
    total = sum(times)
    line = {
        "metric": "surrogate-gradient evaluations/s (10% microcircuit, 200 ms, rate MSE, "
                  "1 GB300)",
        "value": args.steps / total, "unit": "gradients/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "10%% microcircuit (7,717 neurons), %d time steps, %s, gradient "
                               "w.r.t. 64 projection scales and nu"
                               % (n_steps, "trajectory recorded by the forward" if recorded
                                  else "checkpoints every %d steps" % every),
                   "l2": "not flushed; wall-clock per gradient including host marshalling"},
        "loss": loss, "grad_abs_max": float(gs.abs().max()), "grad_nu": float(gn),
        "clocks": clk.summary(),
        # per gradient, recorded: one k_step, one k_adjoint_part, the fold and
        # the reduction; checkpointed: one k_step per segment forward, k_step +
        # k_adjoint_part per segment backward, the fold and the reduction
        "gpu_launches": args.steps * (4 if recorded else 3 * ((n_steps + every - 1) // every) + 2),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--chunk", type=int, default=STEPS_PER_BENCH_STEP,
                    help="time steps per bench step (profiling uses short launches)")
    ap.add_argument("--cpu-skip", type=int, default=500)
    ap.add_argument("--cpu-steps", type=int, default=4000)
    ap.add_argument("--ref-chunk", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 20,000-spike delivery, 4x, batch and gradient keys")
    ap.add_argument("--instances", type=int, default=64, help="instances of --workload batch")
    ap.add_argument("--grad-trace-budget", type=int, default=0,
                    help="--workload grad: trajectory bytes kept by the forward (0: checkpoints)")
    ap.add_argument("--deliver-scale", default="1.0,4.0", help="--workload deliver: scales")
    ap.add_argument("--deliver-spikes", default="25,93,4000,20000", help="--workload deliver: list sizes")
    ap.add_argument("--deliver-tilings", default="0,1,2,3", help="--workload deliver: tilings (4: clusters)")
    ap.add_argument("--workload", default="full",
                    choices=["full", "scale4", "batch", "grad", "deliver", "realtime", "soak"])
    args = ap.parse_args()
    if args.workload == "scale4":
        args.scale = 4.0
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "grad":
        run_grad(args)
    elif args.workload == "deliver":
        run_deliver(args)
    elif args.workload == "realtime":
        run_realtime(args)
    elif args.workload == "soak":
        run_soak(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
