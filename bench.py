"""Benchmark: gate-amplitude updates/s of the state-vector hot path at 30 qubits.

One step = set |0...0>, apply the 30-qubit, 40-layer random circuit (U3 on every
qubit + brickwork CNOT, 1,780 gates, complex64) and read <Z_q> for every qubit.
updates/s = (gates x 2^n) / step time (every gate counts one pass over the state).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fused|plain]
                    [--impl ours|reference] [--no-cpu-baseline]

Under torchrun (N > 1) every rank runs its own replica on its own GPU (the
single-circuit path does not shard); value = all ranks' updates / max time.
--impl reference times the CPU oracle (complex128, host cores) on a bounded
sample of the same workload.
"""
from __future__ import annotations

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

METRIC = "gate-amplitude updates/s and % of HBM roofline at 30 qubits; adjoint grad time"
UNIT = "gate-amplitude updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fused", choices=["fused", "plain"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--layers", type=int, default=40)
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-gates-per-step", type=int, default=8)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint, batch, plain-pass and complex128 measurements")
    return ap.parse_args()


def workload(args):
    from paper_2508_15545_gb300 import workloads as W
    gates = W.random_circuit(args.n, args.layers, W.config_seed(1))
    cfg = {
        "workload": "random circuit, %d qubits, %d layers of U3 on every qubit + brickwork CNOT "
                    "(%d gates), complex64 state from |0...0>, <Z_q> read-out" % (args.n, args.layers, len(gates)),
        "n_qubits": args.n, "layers": args.layers, "gates": len(gates),
        "state_bytes": (1 << args.n) * 8,
        "l2": "inputs larger than L2 (%.1f GiB state vs 129 MB L2)" % ((1 << args.n) * 8 / 2 ** 30),
        "seed": W.config_seed(1),
    }
    return gates, cfg


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Sources that define each kernel class's device code: a committed ncu figure
# stays valid while these files are unchanged.
KERNEL_SOURCES = {
    "plain": ("pair_kernels.cu", "qv_device.cuh"),
}
# The compiled fused passes are generated per pass: their committed ncu
# figure stays valid while the generated sources of the captured workload
# (this circuit recipe at these sizes, default tile size) are unchanged.
GENERATED_CAPTURE = {"fused": {"n": 26, "layers": 40}}


def fp32_peak_tflops(sm_count: int, sm_max_mhz) -> float:
    """FP32 arithmetic peak: 128 FP32 lanes per SM, one FMA (2 operations) per
    lane and clock, at the maximum SM clock (2070 MHz on GB300 when the
    sampler saw none)."""
    mhz = float(sm_max_mhz) if sm_max_mhz else 2070.0
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def source_hash(kernel_class: str, qv=None) -> str:
    h = hashlib.sha256()
    cap = GENERATED_CAPTURE.get(kernel_class)
    if cap is not None:
        # hash of every generated pass source of the captured workload (host only)
        from paper_2508_15545_gb300 import workloads as W
        if qv is None:
            from paper_2508_15545_gb300 import qv
        n = cap["n"]
        gates = W.random_circuit(n, cap["layers"], W.config_seed(1))
        arr = (qv.gates_to_c(gates), len(gates))
        for i in range(qv.qv_plan_info(n, qv.QV_C64, arr)["passes"]):
            h.update(qv.qv_plan_source(n, qv.QV_C64, arr, i).encode())
        return "gen-" + h.hexdigest()[:16]
    csrc = os.path.join(ROOT, "paper_2508_15545_gb300", "csrc")
    for fn in KERNEL_SOURCES.get(kernel_class, ()):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class: str, mode: str, qv=None):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_class)
    if not e or e.get("source_hash") != source_hash(kernel_class, qv):
        return None
    return e.get("dram_bytes_per_launch_scaled")


# ----------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------
def oracle_sample(args, gates, seconds: float, max_gates: int | None = None, threads: int = 1):
    """Applies gates of the workload in order to the full 2^n complex128 state
    with the oracle on `threads` host threads (OpenMP over the pairs of Eq. 5)
    until `seconds` elapse or `max_gates` are done. Returns (gates applied,
    elapsed seconds, state, threads used)."""
    from oracle import oracle
    used = oracle.set_threads(threads)
    psi = oracle.basis(args.n, 0)
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.run(args.n, [gates[done % len(gates)]], psi)
        done += 1
        el = time.perf_counter() - t0
        if (max_gates is not None and done >= max_gates) or (max_gates is None and el >= seconds):
            return done, el, psi, used


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args, gates):
    """The oracle as it stands on the host cores: the first gates of the
    circuit on the full 2^n complex128 state, with one thread and with every
    host core (about args.cpu_seconds / 2 each)."""
    N = 1 << args.n
    half = args.cpu_seconds / 2
    d1, e1, psi, _ = oracle_sample(args, gates, half, threads=1)
    del psi
    dn, en, psi, used = oracle_sample(args, gates, half, threads=host_cores())
    del psi
    return {"value": dn * N / en, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "first %d gates of the circuit on the full 2^%d complex128 state, %d host threads, %.1f s"
                      % (dn, args.n, used, en),
            "single_thread": {"value": d1 * N / e1, "unit": UNIT, "cores": 1,
                              "sample": "first %d gates, one host thread, %.1f s" % (d1, e1)},
            "host_cores_available": host_cores()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    gates, cfg = workload(args)
    from oracle import oracle
    cores = oracle.set_threads(host_cores())
    psi = oracle.basis(args.n, 0)
    N = 1 << args.n
    g = args.ref_gates_per_step
    pos = 0

    def step():
        nonlocal pos
        for _ in range(g):
            oracle.run(args.n, [gates[pos % len(gates)]], psi)
            pos += 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = g * N / (ms / 1e3)
    sample = ("%d gates per step of the %d-gate circuit on the full 2^%d complex128 state, %d host threads"
              % (g, len(gates), args.n, cores))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "host_cores_available": host_cores()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def max_over_ranks(values, device):
    """Max of each value over all ranks: one all-reduce of the timings, the
    only collective of a replica run (no data moves between ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all replicas processed, divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2508_15545_gb300 import qv
    gates, cfg = workload(args)
    mode = qv.QV_MODE_FUSED if args.mode == "fused" else qv.QV_MODE_PLAIN
    cfg["mode"] = args.mode
    cfg["parallelism"] = "replicas%d" % world if world > 1 else "single GPU"
    garr = qv.gates_to_c(gates)
    ng = len(gates)
    plan_cost = None
    if mode == qv.QV_MODE_FUSED:
        cfg["plan"] = qv.qv_plan_info(args.n, qv.QV_C64, (garr, ng), args.tile_bits)
        cfg["tile_bits"] = args.tile_bits or qv.qv_default_tile_bits(args.n, qv.QV_C64)
        plan_cost = qv.qv_plan_cost(args.n, qv.QV_C64, (garr, ng), args.tile_bits)
    N = 1 << args.n

    stream = torch.cuda.current_stream(dev)
    st = qv.StateVector(args.n, qv.QV_C64, stream=stream)
    h = st.h

    def step():
        qv.qv_set_basis(h, 0)
        qv.qv_apply_circuit(h, (garr, ng), mode, args.tile_bits)
        return qv.qv_expect_z(h)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    qv.qv_profile(h, timing=False)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        ez, _ = step()
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    stats = qv.qv_profile_read(h)
    launches = sum(v[0] for v in stats.values())

    # per-class device time: separate timed steps with events around each launch
    qv.qv_profile(h, timing=True)
    for _ in range(2):
        step()
    tstats = qv.qv_profile_read(h)
    qv.qv_profile(h, timing=False)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        qv.qv_profile(h, timing=False)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, gates, mode, args.tile_bits)   # host gate list, marshalled + copied
            qv.qv_expect_z(h)                                       # D2H of <Z_q>
        torch.cuda.synchronize(dev)
        e2e_s = (time.perf_counter() - t0) / args.steps
        h2d, d2h = qv.qv_transfer_bytes(h)
        e2e = {"value_s": e2e_s, "h2d": h2d / args.steps, "d2h": d2h / args.steps}

    ms_max, e2e_max = max_over_ranks([ms, e2e["value_s"] if e2e else 0.0], dev)

    updates = ng * N
    value = whole_job_rate(updates, world, ms_max / 1e3)
    peak, peak_kind = peaks()
    # dominant kernel class by device time
    dom = max(tstats.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms, dbytes) = dom
    achieved = dbytes / (dms / 1e3) / 1e9 if dms > 0 else None
    per_launch = dbytes / dl if dl else None
    roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
            "traffic": ncu_traffic(dname, args.mode, qv),
            "algorithmic_bytes_per_launch": per_launch,
            "avg_launch_ms": dms / dl if dl else None,
            "share_of_step": dms / sum(v[1] for v in tstats.values())}
    if dname == "fused" and plan_cost and dms > 0:
        # A fused pass does many gates per HBM round trip: it is bound by FP32
        # arithmetic when operations / FP32 peak exceed bytes / HBM peak.
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak = fp32_peak_tflops(sm_count, clocks.get("sm_max_mhz"))
        steps_timed = 2
        flops_s = plan_cost["flops"] * steps_timed / (dms / 1e3)
        t_alu = plan_cost["flops"] / (fp32_peak * 1e12)
        t_hbm = plan_cost["bytes"] / (peak * 1e9)
        roof["hbm_frac"] = roof["frac"]
        roof["hbm_achieved_GBps"] = achieved
        roof["alu"] = {"achieved": flops_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                       "frac": flops_s / 1e12 / fp32_peak, "peak_kind": "derived: SMs x 128 FP32 lanes x 2 x max SM clock",
                       "flops_per_launch": plan_cost["flops"] / max(1, cfg["plan"]["passes"])}
        roof["floor_ms_per_step"] = {"hbm": t_hbm * 1e3, "alu": t_alu * 1e3}
        if t_alu > t_hbm:
            roof.update({"bound": "alu", "achieved": flops_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": flops_s / 1e12 / fp32_peak, "peak_kind": roof["alu"]["peak_kind"]})
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roof,
        "kernel_classes": {k: {"launches": v[0] / 2, "ms": v[1] / 2, "GBps": (v[2] / (v[1] / 1e3) / 1e9) if v[1] else None}
                           for k, v in tstats.items() if v[0]},
    }
    if e2e:
        out["e2e"] = {"value": whole_job_rate(updates, world, e2e_max), "unit": UNIT,
                      "h2d_bytes_per_step": int(e2e["h2d"]), "d2h_bytes_per_step": int(e2e["d2h"])}
    if not args.no_extras:
        out["extras"] = extras(args, qv, torch, dev, st.h, gates)
    st.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, gates)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# further measurements of the same build (reported beside the headline value)
# ----------------------------------------------------------------------------
def _timed(torch, dev, fn, reps):
    fn()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize(dev)
    return (time.perf_counter() - t0) / reps * 1e3


def extras(args, qv, torch, dev, h64, gates):
    from paper_2508_15545_gb300 import workloads as W
    peak, _ = peaks()
    res = {}
    N = 1 << args.n
    # 1. per-gate (plain) kernels on the bench state: HBM fraction of one-gate passes
    try:
        sub = gates[:64]
        qv.qv_profile(h64, timing=True)
        qv.qv_apply_circuit(h64, sub, qv.QV_MODE_PLAIN)
        st = qv.qv_profile_read(h64)
        qv.qv_profile(h64, timing=False)
        l, ms, by = st["pair"]
        res["plain_pair_kernel"] = {"gates": l, "ms_per_gate": ms / l, "GBps": by / (ms / 1e3) / 1e9,
                                    "frac_of_measured_hbm": by / (ms / 1e3) / 1e9 / peak,
                                    "algorithmic_bytes_per_gate": by / l,
                                    "note": "U3 passes move 2 x 8 GiB; CNOT passes only the control-1 half"}
    except Exception as e:  # noqa: BLE001
        res["plain_pair_kernel"] = {"error": str(e)}
    # 1b. the fused step with each tile size (the autotuner's choice space)
    try:
        garr = qv.gates_to_c(gates)
        sweep = {}
        for tb in (10, 11, 12):
            if tb > args.n:
                continue

            def one(tb=tb):
                qv.qv_set_basis(h64, 0)
                qv.qv_apply_circuit(h64, (garr, len(gates)), qv.QV_MODE_FUSED, tb)
            sweep["k=%d" % tb] = _timed(torch, dev, one, 2)
        res["tile_size_sweep_ms_per_step"] = sweep
    except Exception as e:  # noqa: BLE001
        res["tile_size_sweep_ms_per_step"] = {"error": str(e)}
    # 1a. qubit remap (Sec. III-E): reverse all qubit positions; SWAPs are relabels inside tiles,
    # so the passes only move data (HBM-bound)
    try:
        perm = list(range(args.n - 1, -1, -1))
        swaps = [W.Gate("swap", p, target2=args.n - 1 - p) for p in range(args.n // 2)]
        rp = qv.qv_plan_info(args.n, qv.QV_C64, swaps)["passes"]
        ms_r = _timed(torch, dev, lambda: qv.qv_permute_qubits(h64, perm), 3)
        gbs = 2.0 * rp * N * 8 / (ms_r / 1e3) / 1e9
        res["qubit_reversal"] = {"passes": rp, "ms": ms_r, "GBps": gbs, "frac_of_measured_hbm": gbs / peak}
    except Exception as e:  # noqa: BLE001
        res["qubit_reversal"] = {"error": str(e)}
    # 1b'. measurement sampling of the bench state: 10^6 shots
    try:
        qv.qv_set_basis(h64, 0)
        qv.qv_apply_circuit(h64, (qv.gates_to_c(gates), len(gates)), qv.QV_MODE_FUSED)
        u = W.SplitMix64(7).uniform(1000000)
        ms_s = _timed(torch, dev, lambda: qv.qv_sample(h64, u), 2)
        res["sampling"] = {"shots": len(u), "ms": ms_s, "shots_per_s": len(u) / (ms_s / 1e3)}
    except Exception as e:  # noqa: BLE001
        res["sampling"] = {"error": str(e)}
    # 1c. the same step with the state in mapped host memory: staged through a device window
    # (one copy in and one out per step) and, for comparison, read and written in place over
    # NVLink-C2C by every pass
    try:
        hh = qv.qv_create(args.n, qv.QV_C64, flags=qv.QV_ALLOC_HOST)
        garr = qv.gates_to_c(gates)

        def host_step(flags=0):
            qv.qv_set_basis(hh, 0)
            qv.qv_apply_circuit(hh, (garr, len(gates)), qv.QV_MODE_FUSED, 0, flags)
        ms_w = _timed(torch, dev, host_step, 2)
        qv.qv_profile(hh, timing=False)
        host_step()
        torch.cuda.synchronize(dev)
        h2d_w, d2h_w = qv.qv_transfer_bytes(hh)
        ms_h = _timed(torch, dev, lambda: host_step(qv.QV_PLAN_HOST_IN_PLACE), 1)
        # the passes of the in-place plan (host states take their own tile size): counted launches
        qv.qv_profile(hh, timing=False)
        host_step(qv.QV_PLAN_HOST_IN_PLACE)
        torch.cuda.synchronize(dev)
        passes = int(qv.qv_profile_read(hh)["fused"][0])
        qv.qv_profile(hh, timing=False)
        res["host_memory_state"] = {
            "window": {"ms_per_step": ms_w, "updates_per_s": len(gates) * N / (ms_w / 1e3),
                       "c2c_bytes_per_step": h2d_w + d2h_w,
                       "note": "the whole state staged into one device window: one copy in, every pass in HBM, "
                               "one copy back"},
            "in_place": {"ms_per_step": ms_h, "updates_per_s": len(gates) * N / (ms_h / 1e3), "passes": passes,
                         "c2c_bytes_per_step": 2 * passes * N * 8,
                         "GBps_over_c2c": 2.0 * passes * N * 8 / (ms_h / 1e3) / 1e9}}
        qv.qv_destroy(hh)
    except Exception as e:  # noqa: BLE001
        res["host_memory_state"] = {"error": str(e)}
    # 1d. the same step with the tensor-core engine (QV_PLAN_TENSOR, 2^12 tiles)
    try:
        garr = qv.gates_to_c(gates)

        def tc_step():
            qv.qv_set_basis(h64, 0)
            qv.qv_apply_circuit(h64, (garr, len(gates)), qv.QV_MODE_FUSED, 12, qv.QV_PLAN_TENSOR)
        ms_tc = _timed(torch, dev, tc_step, 2)
        qv.qv_sync(h64)
        info = qv.qv_plan_info(args.n, qv.QV_C64, (garr, len(gates)), 12, qv.QV_PLAN_TENSOR)
        res["tensor_core_engine"] = {"tile_bits": 12, "ms_per_step": ms_tc,
                                     "updates_per_s": len(gates) * N / (ms_tc / 1e3),
                                     "passes": info["passes"], "stages": info["stages"], "matrix_stages": info["ops"],
                                     "frac_of_measured_hbm": 2.0 * info["passes"] * N * 8 / (ms_tc / 1e3) / 1e9 / peak,
                                     "norm2_after": qv.qv_norm2(h64)}
    except Exception as e:  # noqa: BLE001
        res["tensor_core_engine"] = {"error": str(e)}
    # 1e. end to end through the API: the first call of a new circuit structure
    # (planning + NVRTC of every pass + run), and a variational loop (new angles
    # every step: planning again, compiled passes reused, coefficients uploaded)
    try:
        g41 = W.random_circuit(args.n, args.layers + 1, W.config_seed(1, 41))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        qv.qv_set_basis(h64, 0)
        qv.qv_apply_circuit(h64, g41, qv.QV_MODE_FUSED)
        qv.qv_expect_z(h64)
        first_ms = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        qv.qv_set_basis(h64, 0)
        qv.qv_apply_circuit(h64, g41, qv.QV_MODE_FUSED)
        qv.qv_expect_z(h64)
        again_ms = (time.perf_counter() - t0) * 1e3
        steps_v = 3
        t0 = time.perf_counter()
        for v in range(steps_v):
            gv = W.random_circuit(args.n, args.layers, W.config_seed(1, 500 + v))   # same structure, new angles
            qv.qv_set_basis(h64, 0)
            qv.qv_apply_circuit(h64, gv, qv.QV_MODE_FUSED)
            qv.qv_expect_z(h64)
        var_ms = (time.perf_counter() - t0) * 1e3 / steps_v
        res["e2e_variants"] = {
            "first_call_new_structure_ms": first_ms,
            "same_call_again_ms": again_ms,
            "first_call_note": "%d-layer circuit (%d gates) never planned or compiled in this process: planning, "
                               "NVRTC of every pass, run, <Z_q> read-out" % (args.layers + 1, len(g41)),
            "variational_ms_per_step": var_ms,
            "variational_updates_per_s": len(gates) * N / (var_ms / 1e3),
            "variational_note": "new angles every step (same structure): the plan is made again, the compiled "
                                "passes are reused, coefficients go to the kernels as parameters"}
    except Exception as e:  # noqa: BLE001
        res["e2e_variants"] = {"error": str(e)}
    # 2. complex128 rerun of the bench circuit and its distance to the complex64 result
    try:
        free, _ = torch.cuda.mem_get_info(dev)
        if free > (16 << args.n) + (4 << 30):
            h128 = qv.qv_create(args.n, qv.QV_C128)
            garr = qv.gates_to_c(gates)

            def run128():
                qv.qv_set_basis(h128, 0)
                qv.qv_apply_circuit(h128, (garr, len(gates)), qv.QV_MODE_FUSED)
            ms128 = _timed(torch, dev, run128, 1)
            qv.qv_set_basis(h64, 0)
            qv.qv_apply_circuit(h64, (garr, len(gates)), qv.QV_MODE_FUSED)
            err = qv.qv_distance(h64, h128)
            res["complex128_rerun"] = {"ms_per_step": ms128, "updates_per_s": len(gates) * N / (ms128 / 1e3),
                                       "l2_distance_c64_vs_c128": err, "norm2_c128": qv.qv_norm2(h128)}
            qv.qv_destroy(h128)
    except Exception as e:  # noqa: BLE001
        res["complex128_rerun"] = {"error": str(e)}
    # 3. adjoint gradient: 26-qubit ansatz, 16 layers (832 parameters)
    try:
        n_a, layers_a = 26, 16
        ga, npar = W.ansatz_circuit(n_a, layers_a, W.config_seed(3))
        terms = W.ansatz_hamiltonian(n_a)
        ha = qv.qv_create(n_a, qv.QV_C64)
        garr = qv.gates_to_c(ga)

        def grad(sweep=qv.QV_SWEEP_AUTO):
            qv.qv_set_basis(ha, 0)
            return qv.qv_adjoint_grad(ha, (garr, len(ga)), terms, npar, sweep_mode=sweep)

        def energy():
            qv.qv_set_basis(ha, 0)
            qv.qv_apply_circuit(ha, (garr, len(ga)))
            return qv.qv_expect_pauli(ha, terms)
        ms_g = _timed(torch, dev, grad, 3)
        ms_g_plain = _timed(torch, dev, lambda: grad(qv.QV_SWEEP_PER_GATE), 1)
        ms_g_tiles = _timed(torch, dev, lambda: grad(qv.QV_SWEEP_TILES), 2)
        ms_e = _timed(torch, dev, energy, 2)
        g_t, _ = grad()
        g_p, _ = grad(qv.QV_SWEEP_PER_GATE)
        qv.qv_profile(ha, timing=True)
        grad()
        pst = qv.qv_profile_read(ha)
        qv.qv_profile(ha, timing=False)
        la, msa, bya = pst["adjoint"]
        res["adjoint_grad"] = {"workload": "ansatz 26 qubits, 16 layers of RY, RZ, CZ ring (1248 gates), "
                                           "832 parameters, H = sum ZZ + 0.5 sum X, complex64, FP64 reductions",
                               "ms_per_gradient": ms_g, "ms_per_energy": ms_e,
                               "reverse_sweep": "compiled passes over psi and lambda",
                               "ms_per_gradient_shared_memory_tiles_sweep": ms_g_tiles,
                               "ms_per_gradient_per_gate_sweep": ms_g_plain,
                               "speedup_vs_per_gate_sweep": ms_g_plain / ms_g,
                               "max_abs_diff_vs_per_gate_sweep": float(max(abs(a - b) for a, b in zip(g_t, g_p))),
                               "param_shift_estimate_ms": 2 * npar * ms_e,
                               "speedup_vs_param_shift": 2 * npar * ms_e / ms_g,
                               "reverse_sweep_GBps": bya / (msa / 1e3) / 1e9 if msa else None,
                               "reverse_sweep_frac_of_measured_hbm": (bya / (msa / 1e3) / 1e9 / peak) if msa else None}
        qv.qv_destroy(ha)
    except Exception as e:  # noqa: BLE001
        res["adjoint_grad"] = {"error": str(e)}
    # 3b. size sweep: the random-circuit recipe at 16..30 qubits (20 layers; 40 at five sizes),
    # fused complex64, default tile size; the oracle on every host core beside it
    try:
        from oracle import oracle as O
        othreads = O.set_threads(host_cores())
        sweep = []
        hs = None
        for n_s, layers_s in [(n, 20) for n in range(16, 31)] + [(n, 40) for n in (16, 20, 24, 28, 30)]:
            if n_s > args.n:
                continue
            gs = W.random_circuit(n_s, layers_s, W.config_seed(0, n_s))
            arr = (qv.gates_to_c(gs), len(gs))
            hs = qv.qv_create(n_s, qv.QV_C64)

            def one():
                qv.qv_set_basis(hs, 0)
                qv.qv_apply_circuit(hs, arr, qv.QV_MODE_FUSED)
            ms_s = _timed(torch, dev, one, 3 if n_s < 28 else 1)
            passes = qv.qv_plan_info(n_s, qv.QV_C64, arr)["passes"]
            row = {"n": n_s, "layers": layers_s, "gates": len(gs), "ms": ms_s,
                   "updates_per_s": len(gs) * (1 << n_s) / (ms_s / 1e3), "passes": passes,
                   "frac_of_measured_hbm": 2.0 * passes * (8 << n_s) / (ms_s / 1e3) / 1e9 / peak}
            qv.qv_destroy(hs)
            hs = None
            # the oracle: the whole circuit up to 22 qubits, else its first 8 gates
            ng_o = len(gs) if n_s <= 22 else 8
            psi = O.basis(n_s, 0)
            t0 = time.perf_counter()
            O.run(n_s, gs[:ng_o], psi)
            el = time.perf_counter() - t0
            del psi
            row["oracle_updates_per_s"] = ng_o * (1 << n_s) / el
            row["oracle_sample"] = "%s on %d host threads" % ("whole circuit" if ng_o == len(gs) else "first 8 gates",
                                                               othreads)
            sweep.append(row)
        res["size_sweep"] = sweep
    except Exception as e:  # noqa: BLE001
        res["size_sweep"] = {"error": str(e)}
    # 4. batched ansatz: 256 parameter sets x 20 qubits, 12 layers, <H> per set, one graph
    try:
        nb, lb, cnt = 20, 12, 256
        circuits = [W.ansatz_circuit(nb, lb, W.config_seed(2, c), sigma=0.5)[0] for c in range(cnt)]
        terms = W.ansatz_hamiltonian(nb)
        hs = [qv.qv_create(nb, qv.QV_C64) for _ in range(cnt)]
        b = qv.Batch(list(zip(hs, circuits)), terms)
        ms_b = _timed(torch, dev, b.run, 3)
        nga = sum(len(c) for c in circuits)
        # the same work one circuit at a time through the single-state fused path
        sub = 16
        carrs = [qv.gates_to_c(c) for c in circuits[:sub]]

        def one_by_one():
            for hh, ca, c in zip(hs[:sub], carrs, circuits[:sub]):
                qv.qv_set_basis(hh, 0)
                qv.qv_apply_circuit(hh, (ca, len(c)))
                qv.qv_expect_pauli(hh, terms)
        ms_seq = _timed(torch, dev, one_by_one, 1) * cnt / sub
        res["batch_ansatz"] = {"workload": "256 parameter sets, 20-qubit ansatz, 12 layers (720 gates each), "
                                           "<H> per set, one CUDA graph: every set on its own compiled passes over 16 side streams",
                               "ms_per_batch": ms_b, "updates_per_s": nga * (1 << nb) / (ms_b / 1e3),
                               "one_by_one_estimate_ms": ms_seq, "speedup_vs_one_by_one": ms_seq / ms_b}
        b.close()
        for hh in hs:
            qv.qv_destroy(hh)
    except Exception as e:  # noqa: BLE001
        res["batch_ansatz"] = {"error": str(e)}
    # 5. uneven batch: 64 random circuits, 16..28 qubits, depth 10..60, in one graph: the
    # members that fill the GPU alone on their own compiled passes, the rest in one
    # persistent launch per tile size
    try:
        spec = W.uneven_batch(64, W.config_seed(4))
        circs = [W.random_circuit(n_u, d_u, s_u) for n_u, d_u, s_u in spec]
        hs_u = [qv.qv_create(n_u, qv.QV_C64) for n_u, _, _ in spec]
        t0 = time.perf_counter()
        bu = qv.Batch(list(zip(hs_u, circs)))
        create_s = time.perf_counter() - t0
        ms_u = _timed(torch, dev, bu.run, 2)
        upd = sum(len(c) * (1 << n_u) for c, (n_u, _, _) in zip(circs, spec))
        groups = bu.info()
        res["uneven_batch"] = {"workload": "64 random circuits, qubits uniform in [16, 28], depth uniform in [10, 60], "
                                           "complex64", "ms_per_batch": ms_u, "updates_per_s": upd / (ms_u / 1e3),
                               "create_s": create_s,
                               "tile_bits_per_qubits": {str(g["qubits"]): g["tile_bits"] for g in groups},
                               "members_on_own_passes": sum(1 for g in groups if g["compiled"] == 2),
                               "queued_groups": [g for g in groups if g["compiled"] != 2]}
        bu.close()
        for hh in hs_u:
            qv.qv_destroy(hh)
    except Exception as e:  # noqa: BLE001
        res["uneven_batch"] = {"error": str(e)}
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
