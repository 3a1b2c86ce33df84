"""Benchmark of the GB300 DA-FMM (Coulomb potential + field).

One step = one dafmm_eval (P2M -> M2M -> M2L -> L2L -> L2P + P2P, the whole hot path) over
the resident tree of the workload: N = 1,000,000 particles uniform in the unit cube,
charges U[-1,1], uniform octree of depth 5, expansion order p = 8, seed 2002.

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent replica of
the workload on its own GPU (independent solves shard with no data exchange); the value
is the total particles of all ranks divided by the slowest rank's time.

--impl reference times the CPU oracle (oracle/, plain C, all host cores): each step is one
full oracle solve of the same workload (same tree and order, every particle), nothing
extrapolated.
"""
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

METRIC = "particles/s at rel err <=1e-7 (N=1M, p=8); served solves/s + p50/p99 latency"
UNIT = "particles/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the M2L kernel on
# this workload, from one ncu capture of that kernel; valid while the kernel's source files
# hash to the recorded value, reported as null otherwise
M2L_TRAFFIC = {"fp32": (25.4e6, "eef784baa41f372b")}
M2L_SOURCES = ("paper_2508_02626_gb300/csrc/tc_common.cuh", "paper_2508_02626_gb300/csrc/tc_ops.cu")
# the same for the near-field kernel k_leaf<float> (its source: fmm_order.cuh)
LEAF_TRAFFIC = {"fp32": (117.8e6, "9648eb1373fac813")}
LEAF_SOURCES = ("paper_2508_02626_gb300/csrc/fmm_order.cuh",)


def sources_hash(files):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def m2l_traffic(precision):
    rec = M2L_TRAFFIC.get(precision)
    if rec is None:
        return None
    return rec[0] if sources_hash(M2L_SOURCES) == rec[1] else None


def leaf_traffic(precision):
    rec = LEAF_TRAFFIC.get(precision)
    if rec is None or rec[0] is None:
        return None
    return rec[0] if sources_hash(LEAF_SOURCES) == rec[1] else None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_fma_peak_tflops(sm_mhz):
    """FP32 FMA peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def rotation_madds_per_pair(p, harm=True):
    """Multiply-adds per well-separated pair of the M2L by rotation (Sec. 3.4) at order p: two
    substitutions about x (output (a, b, c) takes b + c + 1 terms), two about z (a + b + 1
    terms) and the axial Eq. 5 matrix (column (a, b, c) reaches row (a', b', c') when b' >= b,
    c' >= c and both differences are even).  harm: the harmonic form (DAFMM_OPT_M2L_HARMONIC,
    default) computes only the outputs of z exponent <= 1 and restores the others before the
    last x-step, two multiply-adds each."""
    C = [(a, b, n - a - b) for n in range(p + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]
    out = [k for k in C if not harm or k[2] <= 1]
    sx = sum(b + c + 1 for a, b, c in out)
    sz = sum(a + b + 1 for a, b, c in out)
    ax = sum(1 for (_, b2, c2) in out for (_, b, c) in C
             if b2 >= b and c2 >= c and (b2 - b) % 2 == 0 and (c2 - c) % 2 == 0)
    restored = 2 * sum(1 for k in C if k[2] > 1) if harm else 0
    return 2 * sx + 2 * sz + ax + restored


def near_field_interactions(x, dom, depth):
    """Pairwise interactions (i != j) of a uniform tree's near field: every particle with every
    other particle of its own leaf and of the adjacent leaves; leaves from the library's box
    rule (21-bit integer coordinates, clamped, shifted down to the leaf level)."""
    s = 1 << depth
    k21 = np.clip(np.floor((np.asarray(x) - np.asarray(dom[:3])) * (2.0 ** 21 / dom[3])), 0, 2 ** 21 - 1)
    k = k21.astype(np.int64) >> (21 - depth)
    cnt = np.zeros((s, s, s), dtype=np.int64)
    np.add.at(cnt, (k[:, 0], k[:, 1], k[:, 2]), 1)
    pad = np.pad(cnt, 1)
    nb = sum(pad[1 + a:1 + a + s, 1 + b:1 + b + s, 1 + c:1 + c + s]
             for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    return int((cnt * nb).sum()) - len(x)


def near_field_roofline(x, dom, depth, leaf_ms, sm_mhz, measured=None):
    """Roofline of the FP32 near-field kernel (P2P over the 27 neighbour leaves; its launch
    also runs L2P): 18 FP32 flops and one rsqrt per interaction (3 differences, r^2 in 5, q/r,
    1/r^2, q/r^3, the potential sum and 3 field FMAs) against the FP32 FMA peak, and
    rsqrt_frac against the rsqrt rate.  With `measured` (the probes of dafmm_probe_peak:
    {"fp32_tflops": the faster of scalar and packed FMA, "rsqrt_per_s": ...}) the peaks are the
    measured ones; the figures from unit counts and clock (152 SMs x 128 FP32 lanes x 2 flops,
    16 MUFU results per SM and clock) are reported beside them."""
    try:
        inter = near_field_interactions(x, dom, depth)
        flops = 18.0 * inter
        sec = leaf_ms / 1e3
        derived = fp32_fma_peak_tflops(sm_mhz)
        derived_rsqrt = 152 * 16 * sm_mhz * 1e6
        if measured:
            peak, rsq = measured["fp32_tflops"], measured["rsqrt_per_s"]
            src = "measured (dafmm_probe_peak: FP32 FMA %.1f TFLOP/s, rsqrt %.3e/s)" % (peak, rsq)
        else:
            peak, rsq = derived, derived_rsqrt
            src = "FP32 FMA = 152 SMs x 128 lanes x 2 flops x %.0f MHz (unit counts and clock)" % sm_mhz
        ach = flops / sec / 1e12
        return {"bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "kernel": "near field k_leaf<float> (P2P over the 27 neighbour leaves, plus L2P; leaf phase time)",
                "algorithmic": "18 FP32 flops + 1 rsqrt per interaction (i != j): %d interactions = %.3e flops"
                               % (inter, flops),
                "peak_source": src,
                "rsqrt_frac": round(inter / sec / rsq, 4),
                "peak_derived": round(derived, 3), "frac_of_derived": round(ach / derived, 4),
                "rsqrt_frac_of_derived": round(inter / sec / derived_rsqrt, 4)}
    except Exception as e:  # the bench line must not be lost to this extra key
        return {"error": repr(e)}


def bench_peaks(device):
    """Unit rates of the GPU measured by the library's probes (dafmm_probe_peak), with the SM
    clock sampled while they run: FP32 FMA (scalar, packed FP32x2), FP64 FMA, MUFU rsqrt, and
    tcgen05 MMA of kind tf32 and f16 (M=128, N=256, one CTA per SM)."""
    import torch

    from paper_2508_02626_gb300 import binding as B
    try:
        uuid = str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        uuid = None
    ck = ClockSampler(device, uuid)
    ck.start()
    out = {}
    try:
        for kind in ("ffma", "ffma2", "dfma", "rsqrt", "mma_tf32", "mma_f16"):
            rate, ms = B.dafmm_probe_peak(device, kind)
            unit = "results/s" if kind == "rsqrt" else "TFLOP/s"
            out[kind] = {"rate": rate if kind == "rsqrt" else round(rate / 1e12, 3), "unit": unit,
                         "ms": round(ms, 3)}
    finally:
        out["clocks"] = ck.stop()
    return out


# clock-event reason bits of NVML (nvml.h) and the names the clock record uses for them
NVML_REASONS = ((0x8, "hw_slowdown"), (0x40, "hw_thermal_slowdown"), (0x20, "sw_thermal_slowdown"),
                (0x4, "sw_power_cap"))
SMI_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def summarise_clocks(nvml_samples, smi_lines):
    """One clock record from both samplers.  nvml_samples: (sm MHz, max sm MHz, reason bits or
    None); smi_lines: nvidia-smi CSV rows of ClockSampler.FIELDS.  The median SM clock and the
    sample count come from NVML when it gave samples (denser), else from nvidia-smi; the
    reasons are those either source saw active."""
    sm_n, smax_n, reasons = [], [], set()
    for clk, mx, bits in nvml_samples:
        sm_n.append(float(clk))
        smax_n.append(float(mx))
        if bits is not None:
            reasons.update(nm for bit, nm in NVML_REASONS if bits & bit)
    sm_s, smax_s = [], []
    for ln in smi_lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 8:
            continue
        try:
            sm_s.append(float(parts[0]))
            smax_s.append(float(parts[1]))
        except ValueError:
            continue
        reasons.update(nm for nm, v in zip(SMI_REASONS, parts[4:8]) if v.lower().startswith("active"))
    sm, smax, src = (sm_n, smax_n, "nvml") if sm_n else (sm_s, smax_s, "nvidia-smi")
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm), "source": src if sm else None,
            "nvidia_smi_samples": len(sm_s)}


class ClockSampler:
    """SM clock and clock-event reasons while the timed region runs: NVML queried every 5 ms
    from a thread (read-only calls into libnvidia-ml), and nvidia-smi every 200 ms beside it."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, uuid=None):
        self.gpu = gpu_index
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None
        self.nvml = None
        self.samples = []
        self.done = threading.Event()
        self.poller = None

    def _nvml_open(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            ok = False
            if self.uuid:
                u = self.uuid if self.uuid.startswith("GPU-") else "GPU-" + self.uuid
                ok = lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
            if not ok:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) == 0
            if not ok:
                lib.nvmlShutdown()
                return None
            reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            return lib, h, reasons
        except Exception:
            return None

    def _nvml_sample(self):
        import ctypes
        lib, h, reasons = self.nvml
        clk, mx, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) != 0:  # 1 = NVML_CLOCK_SM
            return
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0:
            return
        ok = reasons(h, ctypes.byref(bits)) == 0
        self.samples.append((clk.value, mx.value, bits.value if ok else None))

    def _poll(self):
        while not self.done.wait(0.005):
            self._nvml_sample()

    def start(self):
        self.nvml = self._nvml_open()
        if self.nvml is not None:
            self._nvml_sample()
            self.poller = threading.Thread(target=self._poll, daemon=True)
            self.poller.start()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self._nvml_sample()
            self.done.set()
            self.poller.join(timeout=5)
            self.nvml[0].nvmlShutdown()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)
        if self.nvml is None and self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvml and nvidia-smi unavailable"],
                    "samples": 0}
        return summarise_clocks(list(self.samples), list(self.lines))


def max_over_ranks(ms, world, device):
    """The slowest rank's time (every rank gets it); a plain value when running alone."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(units_per_rank, steps, world, max_ms):
    """Whole-job rate of independent replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * steps * world / (max_ms / 1e3)


def m2l_pairs_level(level):
    """Well-separated pairs at one level of a full uniform tree (children of adjacent parents
    that are not adjacent themselves, counted axis by axis)."""
    s = 1 << level
    cand = (3 * (s // 2) - 2) * 4
    near = 3 * s - 2
    return cand ** 3 - near ** 3


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_2508_02626_gb300 import binding as B
    from paper_2508_02626_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = W.C2
    x, q, dom = W.make(cfg)
    n, p, depth = cfg["n"], cfg["order"], cfg["uniform_depth"]
    prec = B.PRECISIONS[args.precision]
    B.load()
    ctx = B.Context(local)
    stream = torch.cuda.Stream(device=dev)
    xt = torch.from_numpy(x).to(dev)
    qt = torch.from_numpy(q).to(dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    E = torch.empty((n, 3), dtype=torch.float64, device=dev)
    tree = ctx.build_tree(xt, qt, domain=dom, uniform_depth=depth, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    B.dafmm_set_profiling(ctx.h, True)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            tree.eval(p, phi, E, precision=prec, stream=stream)
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(local, uuid)
    clocks.start()
    times, phases = [], []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps (outside the timed events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree.eval(p, phi, E, precision=prec, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            phases.append(B.dafmm_last_phase_ms(ctx.h))
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = float(np.sum(times))
    total_ms = max_over_ranks(total_ms, world, dev)
    value = replica_throughput(n, args.steps, world, total_ms)
    ph = {k: float(np.mean([d[k] for d in phases])) for k in phases[0]}

    # the other precision modes on the same tree (a few steps each), for comparison
    modes = {}
    mode_results = {}
    if not args.no_modes:
        for mname in ("mixed", "fp64", "fp64_dense_m2l", "fp32_tf32_m2l", "ff"):
            if mname == args.precision or (args.modes and mname not in args.modes.split(",")):
                continue
            # fp64 uses the M2L by rotation (Sec. 3.4, the default from p = 4); fp64_dense_m2l
            # the dense matrix per displacement, for comparison; fp32_tf32_m2l the FP32 mode with
            # TF32 instead of F16 split operands in M2L -- against MIXED (the same M2L, FP64
            # M2M/L2L and storage) it shows what the FP32 shifts cost in accuracy; ff the
            # float-float mode (FP64-level accuracy on the FP32 pipe)
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_ROTATION, 0 if mname == "fp64_dense_m2l" else -1)
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_F16, 0 if mname == "fp32_tf32_m2l" else 1)
            mp = B.PRECISIONS["fp64" if mname.startswith("fp64") else ("fp32" if mname.startswith("fp32") else mname)]
            ksteps = 2 if mname.startswith("fp64") else 5
            with torch.cuda.stream(stream):
                tree.eval(p, phi, E, precision=mp, stream=stream)
                ms = []
                for _ in range(ksteps):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    tree.eval(p, phi, E, precision=mp, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
            modes[mname] = {"value": n / (float(np.mean(ms)) / 1e3), "ms_per_step": float(np.mean(ms)),
                            "phases_ms": {k: round(v, 4) for k, v in B.dafmm_last_phase_ms(ctx.h).items()
                                          if k != "launches"}}
            mode_results[mname] = (phi.cpu().numpy(), E.cpu().numpy())
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_ROTATION, -1)
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_F16, 1)
        # back to the headline mode for the accuracy sample
        with torch.cuda.stream(stream):
            tree.eval(p, phi, E, precision=prec, stream=stream)
        stream.synchronize()

    # end to end through the public API with host buffers: build_tree + eval per step,
    # host->device copies of the step's inputs and device->host copies of the results
    xp = torch.from_numpy(x).pin_memory()
    qp = torch.from_numpy(q).pin_memory()
    phi_h = torch.empty(n, dtype=torch.float64).pin_memory()
    E_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    e2e_value = e2e_plain = None
    if not args.no_e2e:
        def e2e_rate(c):
            for _ in range(2):
                tr = c.build_tree(xp, qp, domain=dom, uniform_depth=depth, stream=stream)
                tr.eval(p, phi_h, E_h, precision=prec, stream=stream)
                tr.free()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                tr = c.build_tree(xp, qp, domain=dom, uniform_depth=depth, stream=stream)
                tr.eval(p, phi_h, E_h, precision=prec, stream=stream)
                tr.free()
            torch.cuda.synchronize()
            return n * e2e_steps / (time.perf_counter() - t0)

        # a pooled context carves every tree and scratch array out of one reservation, so
        # freeing a tree between steps never synchronises the device
        pool = B.Context(local, pool_bytes=4 << 30)
        e2e_value = e2e_rate(pool) * world
        pool.close()
        e2e_plain = e2e_rate(ctx) * world

    # measured unit rates (FP32 / FP64 / MUFU / tcgen05 TF32 and F16), after the timed region
    probes = None
    if not args.no_peaks:
        try:
            probes = bench_peaks(local)
        except Exception as e:  # the bench line must not be lost to this extra key
            probes = {"error": repr(e)}
    measured_alu = None
    if probes and "ffma" in probes:
        measured_alu = {"fp32_tflops": max(probes["ffma"]["rate"], probes["ffma2"]["rate"]),
                        "rsqrt_per_s": probes["rsqrt"]["rate"], "fp64_tflops": probes["dfma"]["rate"]}

    # the FP64 mode's two dominant kernels against the measured FP64 FMA rate: the M2L by
    # rotation (its multiply-adds, Sec. 3.4) and the leaf kernel (18 FP64 flops and one
    # rsqrt per near-field interaction; its launch also runs L2P)
    if measured_alu and "fp64" in modes and p >= 4:
        pf = measured_alu["fp64_tflops"]
        ph64 = modes["fp64"]["phases_ms"]
        pairs64 = sum(m2l_pairs_level(l) for l in range(2, depth + 1))
        rot_fl = 2.0 * rotation_madds_per_pair(p) * pairs64
        inter = near_field_interactions(x, dom, depth)
        modes["fp64"]["rooflines"] = {
            "peak_fp64_tflops": round(pf, 4), "peak_source": "measured (dafmm_probe_peak, FP64 FMA)",
            "m2l_rotation": {"algorithmic_flops": rot_fl, "ms": ph64["m2l"],
                             "achieved": round(rot_fl / (ph64["m2l"] / 1e3) / 1e12, 4),
                             "frac": round(rot_fl / (ph64["m2l"] / 1e3) / 1e12 / pf, 4)},
            "leaf": {"algorithmic_flops": 18.0 * inter, "interactions": inter, "ms": ph64["leaf"],
                     "achieved": round(18.0 * inter / (ph64["leaf"] / 1e3) / 1e12, 4),
                     "frac": round(18.0 * inter / (ph64["leaf"] / 1e3) / 1e12 / pf, 4)}}

    peaks, peak_src = load_peaks()
    nc = (p + 1) * (p + 2) * (p + 3) // 6
    pairs_all = sum(m2l_pairs_level(l) for l in range(2, depth + 1))
    flops = 2.0 * nc * nc * pairs_all
    m2l_s = ph["m2l"] / 1e3
    achieved = flops / m2l_s / 1e12
    f16 = args.precision == "fp32"  # the FP32 mode's M2L runs on F16 split operands (the default)
    rot = args.precision == "fp64" and p >= 4  # the FP64 default M2L from p = 4: by rotation
    if args.precision == "fp64":
        peak, bound = 1.25, "alu"
        peak_note = "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"
        if measured_alu:
            peak = measured_alu["fp64_tflops"]
            peak_note = "FP64 FMA measured by dafmm_probe_peak (%.3f TFLOP/s; nominal 1.25)" % peak
        executed = None
        if rot:
            flops = 2.0 * rotation_madds_per_pair(p) * pairs_all
            achieved = flops / m2l_s / 1e12
    else:
        if f16:
            # F16 operands: dense F16 tensor peak = the measured BF16 burst peak (same nominal rate)
            peak, bound = peaks["bf16_tflops"], "tensor"
            peak_note = "F16 = %s BF16 %.1f TFLOP/s (same nominal dense rate)" % (peak_src, peaks["bf16_tflops"])
        else:
            # TF32 tensor peak = measured BF16 burst peak x the nominal TF32/BF16 ratio 1/2
            peak, bound = peaks["bf16_tflops"] / 2.0, "tensor"
            peak_note = "TF32 = %s BF16 %.1f TFLOP/s x 1/2 (nominal ratio)" % (peak_src, peaks["bf16_tflops"])
        # the FP32 mode's F16 M2L runs in the harmonic basis (DAFMM_OPT_M2L_HARMONIC, default):
        # rows and columns of the contraction are the (p + 1)^2 free coefficients
        nk = (p + 1) ** 2  # both operand forms run in the harmonic basis by default
        npt = (nk + 15) // 16 * 16
        if npt > 192:
            npt = 2 * (((npt // 2) + 15) // 16 * 16)
        klen = (nk + 15) // 16 * 16 if f16 else (nk + 7) // 8 * 8  # operand row length (MMA K)
        tiles = 0
        for l in range(2, depth + 1):
            S = 1 << (l - 1)
            bx = min(S, 128); by = min(S, 128 // bx); bz = max(1, min(S, 128 // (bx * by)))
            tiles += 8 * (S // bx) * (S // by) * (S // bz)
        executed = tiles * 189 * 3 * 2.0 * 128 * npt * klen / m2l_s / 1e12
    roofline = {"bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": m2l_traffic(args.precision), "traffic_unit": "bytes per launch",
                "kernel": ("M2L contraction (tcgen05 kind::f16 k_tc, all levels, one launch)" if f16 else
                           "M2L contraction (tcgen05 kind::tf32 k_tc, all levels, one launch)") if bound == "tensor"
                else ("M2L by rotation (k_m2l_rot, FP64 pipe, all levels)" if rot else
                      "M2L (SIMT FP64 k_m2l, all levels)"),
                "algorithmic": ("2 x %d multiply-adds per well-separated pair (4 rotations + axial Eq. 5, "
                                "harmonic form: outputs of z exponent <= 1, the others restored): %.3e flops"
                                % (rotation_madds_per_pair(p), flops)) if rot else
                               ("2 ncoef^2 flops per well-separated pair: %.3e flops (the dense M2L of Eq. 5; "
                                "computed in the harmonic basis, 2 (p+1)^4 = %.3e flops, plus the expansion of "
                                "the locals, inside the timed phase)" % (flops, 2.0 * (p + 1) ** 4 * pairs_all)
                                if bound == "tensor" else "2 ncoef^2 flops per well-separated pair: %.3e flops" % flops),
                "achieved_harmonic": (round(2.0 * (p + 1) ** 4 * pairs_all / m2l_s / 1e12, 3)
                                      if bound == "tensor" else None),
                "frac_harmonic": (round(2.0 * (p + 1) ** 4 * pairs_all / m2l_s / 1e12 / peak, 4)
                                  if bound == "tensor" else None),
                "executed_tflops": None if executed is None else round(executed, 3),
                "executed_frac": None if executed is None else round(executed / peak, 4),
                "peak_source": peak_note}

    near_roof = None
    if args.precision != "fp64":
        near_roof = near_field_roofline(x, dom, depth, ph["leaf"], peaks.get("sm_max_mhz", 2070.0), measured_alu)
        if "error" in near_roof:
            near_roof = None
        else:
            near_roof["traffic"] = leaf_traffic(args.precision)
            near_roof["traffic_unit"] = "bytes per launch"
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64 (M2L tf32x3)",
                  "fp32": "f32 (M2L f16x3 scaled split products, M2M/L2L tf32x3)"}[args.precision],
        "data": "synthetic (seeded uniform, PCG64 seed 2002)",
        "config": {"workload": "uniform N=1e6, q~U[-1,1], octree depth 5, order p=8, theta=1",
                   "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "phases_ms": {k: round(v, 4) for k, v in ph.items() if k != "launches"},
        "gpu_launches": int(ph["launches"]) * args.steps,
        # `roofline` describes the step's dominant kernel: the near field (k_leaf, about 55% of
        # the FP32 step); the M2L contraction's figures follow under roofline_m2l
        "roofline": near_roof if near_roof is not None else roofline,
        "roofline_m2l": roofline if near_roof is not None else None,
        "peaks": probes,
        "clocks": ck,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 4 * 8,
                "d2h_bytes_per_step": n * 4 * 8, "steps": e2e_steps,
                "includes": "dafmm_build_tree + dafmm_eval from pinned host buffers (pooled context)",
                "value_ordinary_context": e2e_plain},
        "modes": modes,
    }
    phi_host, E_host = phi.cpu().numpy(), E.cpu().numpy()
    # the method's own error against the direct sum as a function of the order (FP64 path, the
    # same tree): which order, if any, reaches the metric's 1e-7 on this workload
    phi_by_order = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        for po in range(2, 11):
            tree.eval(po, phi, None, precision="fp64")
            phi_by_order[po] = phi.cpu().numpy().copy()
    tree.free()
    if world == 1 and not args.no_workloads:
        sections = set(args.sections.split(","))
        if "adaptive" in sections:
            out["adaptive"] = bench_adaptive(ctx, stream, flush, args.adaptive_n,
                                             tuple(args.adaptive_modes.split(",")))
        if "batch" in sections:
            out["batch"] = bench_batch(ctx, stream, flush)
        if "serving" in sections:
            out["serving"] = bench_serving(args.serving_requests)
        if "operators" in sections:
            out["operators"] = bench_operators(ctx)
            out["noalloc"] = bench_noalloc(ctx)
        if "leafsize" in sections:
            out["leaf_size"] = bench_leaf_size(ctx)
        if "paper" in sections:
            out["paper_shape"] = bench_paper_shape(ctx)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["accuracy"] = cpu_baseline(x, q, dom, cfg, phi_host, E_host, phi_by_order,
                                                            mode_results)
        for mname, errs in out["accuracy"].pop("modes", {}).items():
            out["modes"][mname].update(errs)
        a = out["accuracy"]
        # the headline's error beside its value: against the FP64 oracle FMM (same tree and
        # order, all particles) and, with the oracle's own, against the direct sum
        out["config"]["error"] = {k: float("%.3e" % a[k]) for k in (
            "rel_l2_phi_vs_oracle", "rel_l2_field_vs_oracle", "worst_target_field_vs_oracle",
            "rel_l2_phi_vs_direct", "oracle_rel_l2_phi_vs_direct", "rel_l2_field_vs_direct",
            "oracle_rel_l2_field_vs_direct")}
    if "fp64" in out["modes"]:
        out["config"]["fp64_mode_particles_per_s"] = round(out["modes"]["fp64"]["value"])
    if "ff" in out["modes"]:  # the float-float mode: FP64-level agreement with the oracle
        m = out["modes"]["ff"]
        out["config"]["ff_mode"] = {"particles_per_s": round(m["value"])}
        for k in ("rel_l2_phi_vs_oracle", "rel_l2_field_vs_oracle"):
            if k in m:
                out["config"]["ff_mode"][k] = float("%.3e" % m[k])
    ctx.close()
    return out


def timed_evals(tree, p, prec, phi, E, stream, flush, steps):
    import torch
    ms = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree.eval(p, phi, E, precision=prec, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms))


def bench_adaptive(ctx, stream, flush, n_points=None, modes=("mixed", "fp32")):
    """Adaptive octree on clustered data: N = 4e6 in 32 Gaussian clusters, q = +1, s = 64,
    p = 10; MIXED (the workload's stated precision) and FP32.  n_points replaces N (a smaller
    case of the same distribution, for profiling captures)."""
    import torch

    from paper_2508_02626_gb300 import binding as B
    from paper_2508_02626_gb300 import workloads as W
    cfg = dict(W.C3)
    if n_points:
        cfg["n"] = int(n_points)
    x, q, _ = W.make(cfg)
    n, p = cfg["n"], cfg["order"]
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree = ctx.build_tree(xt, qt, domain=None, uniform_depth=-1, max_leaf=cfg["max_leaf"], stream=stream)
    stream.synchronize()
    t0 = time.perf_counter()
    tr2 = ctx.build_tree(xt, qt, domain=None, uniform_depth=-1, max_leaf=cfg["max_leaf"], stream=stream)
    stream.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    tr2.free()
    info = tree.info()
    out = {"workload": "clustered N=%.0e (32 Gaussian clusters, sigma U[0.02,0.1]), q=+1, adaptive s=64, p=10" % n,
           "tree": {k: info[k] for k in ("depth", "leaves", "boxes", "max_per_leaf", "m2l_pairs", "p2p_leaf_pairs")},
           "build_ms": build_ms}
    for mname in modes:
        mp = B.PRECISIONS[mname]
        with torch.cuda.stream(stream):
            tree.eval(p, phi, E, precision=mp, stream=stream)
        ms = timed_evals(tree, p, mp, phi, E, stream, flush, 3)
        out[mname] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                      "phases_ms": {k: round(v, 3) for k, v in B.dafmm_last_phase_ms(ctx.h).items()}}
    tree.free()
    return out


def bench_batch(ctx, stream, flush):
    """Batched launch: 256 independent problems (N log-uniform in [1e3, 1e5], uniform or
    clustered by seed, q U[-1,1]), p = 6, FP32, one forest replayed as one CUDA graph, leaf
    size and near-field tile from the autotuner; against the same problems solved one by one
    in plain FP64."""
    import torch

    from paper_2508_02626_gb300 import autotune as A
    from paper_2508_02626_gb300 import binding as B
    from paper_2508_02626_gb300 import workloads as W
    import oracle as O
    sizes = W.batch_sizes()
    xs, qs = zip(*[W.batch_member(n, kind, seed) for n, kind, seed in sizes])
    offs = np.concatenate([[0], np.cumsum([len(v) for v in qs])]).astype(np.int64)
    x, q = np.concatenate(xs), np.concatenate(qs)
    n, p = int(offs[-1]), 6
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    cache = A.Cache(os.path.join(ROOT, "paper_2508_02626_gb300", "_build", "autotune.json"))  # git-ignored
    tuned = A.tune_forest(ctx, xt, qt, offs, p, "fp32", cache=cache, reps=1)
    s = tuned["max_leaf"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = ctx.build_forest(xt, qt, offs, max_leaf=s, stream=stream)
    stream.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    g = f.graph(p, phi, E, precision="fp32", stream=stream)
    ms = []
    for _ in range(5):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.launch(stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    graph_ms = float(np.mean(ms))
    nodes = g.nodes()
    phi_b = phi.cpu().numpy()
    g.free()
    f.free()
    # the same problems as plain FP64 single solves, one after another (tree per problem at
    # the paper's leaf size for p = 6, host buffers in and out)
    s64 = A.paper_leaf_size(p)
    ph64 = np.zeros(n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(len(sizes)):
        a, b = offs[r], offs[r + 1]
        t = ctx.build_tree(xs[r], qs[r], domain=None, uniform_depth=-1, max_leaf=s64)
        t.eval(p, ph64[a:b], None, precision="fp64")
        t.free()
    seq_s = time.perf_counter() - t0
    # equal accuracy: every problem's batched FP32 and single FP64 results against the direct
    # sum (Eq. 1, the oracle's) on 64 seeded targets of that problem
    rng = np.random.default_rng(4999)
    e32, e64 = [], []
    for r in range(len(sizes)):
        a, b = offs[r], offs[r + 1]
        tg = np.sort(rng.choice(b - a, min(64, b - a), replace=False))
        d_phi, _ = O.direct(xs[r], qs[r], targets=tg)
        rl = lambda u: float(np.sqrt(((u[tg] - d_phi) ** 2).sum() / (d_phi ** 2).sum()))
        e32.append(rl(phi_b[a:b]))
        e64.append(rl(ph64[a:b]))
    e32, e64 = np.array(e32), np.array(e64)
    acc = {"problems": len(sizes), "targets_per_problem": 64,
           "batched_fp32_median": float(np.median(e32)), "batched_fp32_max": float(e32.max()),
           "single_fp64_median": float(np.median(e64)), "single_fp64_max": float(e64.max()),
           "note": "potential, relative L2 against the direct sum; the two forms use their own leaf sizes"}
    # ratios where the FP64 solve has a method error; with its larger leaf size a small problem
    # can be a single leaf there, i.e. a direct sum (error ~1e-16), and a ratio means nothing
    m = e64 > 1e-10
    acc.update({"ratio_median": float(np.median(e32[m] / e64[m])) if m.any() else None,
                "ratio_max": float((e32[m] / e64[m]).max()) if m.any() else None,
                "problems_in_ratio": int(m.sum()),
                "fp64_direct_problems": int((~m).sum()),
                "batched_fp32_max_on_those": float(e32[~m].max()) if (~m).any() else None})
    return {"workload": "256 problems, N log-uniform [1e3,1e5], uniform/clustered by seed, q U[-1,1], p=6",
            "particles": n, "autotuned": {"max_leaf": s, "leaf_warps": tuned["leaf_warps"],
                                          "cached": tuned["cached"]},
            "build_ms": build_ms, "graph_ms": graph_ms, "graph_nodes": nodes,
            "solves_per_s": len(sizes) / (graph_ms / 1e3), "value": n / (graph_ms / 1e3),
            "value_with_build": n / ((graph_ms + build_ms) / 1e3), "unit": UNIT,
            "sequential_fp64": {"value": n / seq_s, "solves_per_s": len(sizes) / seq_s, "seconds": seq_s,
                                "max_leaf": s64, "includes": "build_tree + eval per problem, host buffers"},
            "accuracy_vs_direct": acc}


def bench_serving(requests, fp64_every=4, direct_targets=8):
    """Serving loop on the Poisson request stream (N log-uniform in [1e3, 1e6], p in {4, 6, 8},
    uniform or clustered, q U[-1,1], FP32, s = 64): the first `requests` requests of the
    stream (2000: the whole stream); capacity from a saturated run, then arrivals at 0.5, 0.8
    and 1.0 x capacity, p50/p99 latency from submission to results in the caller's
    page-locked buffers.  Every `fp64_every`-th request is also solved as a plain FP64 single
    solve (build + eval, one after another): that gives the sequential FP64 baseline on the
    same requests and, per served result, its error against the FP64 result over all its
    particles (the FP64 path equals the oracle FMM to 1e-12).  Every served result is also
    compared with the direct sum (Eq. 1, the oracle's) on `direct_targets` seeded targets,
    beside the FP64 result's error on the same targets ("equal accuracy")."""
    import torch

    import oracle as O
    from paper_2508_02626_gb300 import binding as B
    from paper_2508_02626_gb300 import workloads as W
    stream_def = W.poisson_stream()[:requests]
    data = []
    for r in stream_def:
        x, q = W.batch_member(r["n"], r["kind"], r["seed"])
        xp = torch.from_numpy(x).pin_memory()
        qp = torch.from_numpy(q).pin_memory()
        out = (torch.empty(len(q), dtype=torch.float64).pin_memory(),
               torch.empty((len(q), 3), dtype=torch.float64).pin_memory())
        data.append((xp, qp, out, r["order"]))
    total_n = int(sum(len(d[1]) for d in data))
    free, _ = torch.cuda.mem_get_info()
    pool = int(min(0.5 * free, 48 << 30))
    srv = B.Server(torch.cuda.current_device(), pool_bytes=pool, slots=4, max_batch=32, max_job_particles=1 << 21)

    def run(arrivals):
        ids = []
        t0 = time.perf_counter()
        for (xp, qp, out, p), ta in zip(data, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(xp, qp, p, precision="fp32", max_leaf=64, out=out))
        lat = []
        for rid in ids:
            st, _, _, tm = srv.wait(rid, timeout=600.0)
            if st != B.DAFMM_OK:
                raise RuntimeError("served request failed: %d %s" % (st, srv.last_error()))
            lat.append(tm["latency_ms"])
        span = time.perf_counter() - t0
        return lat, span

    # warm: the per-order tables of every order in the stream
    warm = [next(i for i, d in enumerate(data) if d[3] == p) for p in sorted({d[3] for d in data})]
    for i in warm:
        st, _, _, _ = srv.wait(srv.submit(data[i][0], data[i][1], data[i][3], precision="fp32", max_leaf=64,
                                          out=data[i][2]), timeout=600.0)
    lat, span = run([0.0] * len(data))
    capacity = len(data) / span
    out = {"workload": "Poisson stream, first %d requests: N log-uniform [1e3,1e6] (%d particles), p in {4,6,8}, "
                       "uniform/clustered, q U[-1,1], FP32, s=64" % (len(data), total_n),
           "slots": 4, "max_batch": 32, "pool_bytes": pool,
           "saturated": {"solves_per_s": capacity, "particles_per_s": total_n / span,
                         "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))},
           "rates": []}
    gaps = np.array([r["t"] for r in stream_def])
    gaps = gaps - gaps[0]
    for f in (0.5, 0.8, 1.0):
        arr = gaps / gaps[-1] * (len(data) / (f * capacity)) if gaps[-1] > 0 else gaps
        lat, span = run(arr)
        out["rates"].append({"load": f, "offered_solves_per_s": f * capacity, "solves_per_s": len(data) / span,
                             "particles_per_s": total_n / span, "p50_ms": float(np.percentile(lat, 50)),
                             "p99_ms": float(np.percentile(lat, 99))})
    st = srv.stats()
    out["server"] = {k: st[k] for k in ("jobs", "requests_per_job", "peak_running", "peak_bytes")}
    srv.close()
    # the served results stay in the page-locked outputs (from the last run)
    served = [(d[2][0].numpy(), d[2][1].numpy()) for d in data]
    # plain FP64 single solves, one after another, of every fp64_every-th request
    ctx = B.Context(torch.cuda.current_device())
    sample = list(range(0, len(data), fp64_every))
    fp64 = {}
    sample_n = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        xp, qp, _, p = data[i]
        fp64[i] = (np.empty(len(qp)), np.empty((len(qp), 3)))
        t = ctx.build_tree(xp, qp, domain=None, uniform_depth=-1, max_leaf=64)
        t.eval(p, fp64[i][0], fp64[i][1], precision="fp64")
        t.free()
        sample_n += len(qp)
    seq_s = time.perf_counter() - t0
    ctx.close()
    out["sequential_fp64"] = {"requests": len(sample), "particles": sample_n, "particles_per_s": sample_n / seq_s,
                              "solves_per_s": len(sample) / seq_s,
                              "note": "every %d-th request of the same stream, build + eval each" % fp64_every}

    def rel(a, b):
        return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))

    # per served result: against its FP64 solve (all particles) and against the direct sum
    vs64_phi, vs64_E, d_served, d_fp64 = [], [], [], []
    rng = np.random.default_rng(5006)
    for i, d in enumerate(data):
        x, q = d[0].numpy(), d[1].numpy()
        tg = np.sort(rng.choice(len(q), min(direct_targets, len(q)), replace=False))
        dphi, dE = O.direct(x, q, targets=tg)
        d_served.append((rel(served[i][0][tg], dphi), rel(served[i][1][tg], dE)))
        if i in fp64:
            vs64_phi.append(rel(served[i][0], fp64[i][0]))
            vs64_E.append(rel(served[i][1], fp64[i][1]))
            d_fp64.append((rel(fp64[i][0][tg], dphi), rel(fp64[i][1][tg], dE)))
    d_served = np.array(d_served)
    d_fp64 = np.array(d_fp64)
    ds_sub = d_served[sample]

    def summ(v):
        v = np.asarray(v)
        return {"median": float(np.median(v)), "p99": float(np.percentile(v, 99)), "max": float(v.max())}

    out["accuracy"] = {
        "served_vs_fp64_rel_l2": {"requests": len(vs64_phi), "phi": summ(vs64_phi), "field": summ(vs64_E),
                                  "within_fp32_bounds": int(sum(1 for a, b in zip(vs64_phi, vs64_E)
                                                                if a <= 3.8e-6 and b <= 1e-5)),
                                  "bounds": "phi 3.8e-6, field 1e-5 (64 u, 160 u)"},
        "served_vs_direct": {"requests": len(d_served), "targets_per_request": direct_targets,
                             "phi": summ(d_served[:, 0]), "field": summ(d_served[:, 1])},
        "equal_accuracy_vs_direct": {"requests": len(d_fp64),
                                     "served_phi_median": float(np.median(ds_sub[:, 0])),
                                     "fp64_phi_median": float(np.median(d_fp64[:, 0])),
                                     "served_field_median": float(np.median(ds_sub[:, 1])),
                                     "fp64_field_median": float(np.median(d_fp64[:, 1])),
                                     "max_ratio_phi": float((ds_sub[:, 0] / np.maximum(d_fp64[:, 0], 1e-300)).max())}}
    return out


def bench_noalloc(ctx):
    """dafmm_eval_noalloc (FP64, every intermediate in the library's fixed array: it copies the
    operator tables in and regenerates the 343 M2L matrices on every call) beside dafmm_eval FP64
    on the same tree (its tables and matrices made once and kept): wall time per call, the
    stream synchronised after each, 20 calls after 3 warm-up calls."""
    import time

    import torch

    from paper_2508_02626_gb300 import binding as B
    from paper_2508_02626_gb300 import workloads as W
    out = {}
    for n, depth, p in ((10000, 3, 6), (40000, 4, 6)):
        x, q = W.uniform(n, seed=880 + depth)
        tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=W.UNIT_CUBE,
                              uniform_depth=depth)
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        res = {}
        for name, call in (("eval_ms", lambda: tree.eval(p, phi, E, precision="fp64")),
                           ("noalloc_ms", lambda: B.dafmm_eval_noalloc(ctx.h, tree.h, p, phi, E))):
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(20):
                call()
                torch.cuda.synchronize()
            res[name] = round((time.perf_counter() - t0) / 20 * 1e3, 3)
        tree.free()
        out["N=%d depth %d p=%d" % (n, depth, p)] = res
    return out


def bench_operators(ctx):
    """Per-operator cost, the GPU analogue of the paper's operator tables (Tables 2-8): each
    generated operator applied to a batch of random instances (ns per instance, FP64 and
    FP32), the same operators by numerical DA on the GPU (DAFMM_OP_NUMERICAL_DA, FP64) and
    their ratio to the generated FP64 code (the paper's Tables 2-8 ratio on one device), the
    batched M2L contraction inside an evaluation (ns per well-separated pair), and the
    oracle's numerical-DA operator per call on one host core (us)."""
    import torch

    from paper_2508_02626_gb300 import binding as B
    from paper_2508_02626_gb300 import workloads as W
    import oracle as O
    rng = np.random.default_rng(31)
    out = {"note": "GPU: ns per instance of a batch of 2^18 (M2L: per pair inside a uniform N=2^18 depth-4 "
                   "evaluation; gpu_fp64_ns: the dense FP64 M2L, gpu_fp64_rotation_ns: the FP64 M2L by "
                   "rotation, Sec. 3.4); gpu_numerical_da_ns: the same operator by numerical DA on the GPU "
                   "(FP64, one warp per instance, a batch of 2^15..2^10 by order); oracle: us per call of "
                   "its numerical-DA operator, one host core"}
    count = 1 << 18
    for p in (2, 4, 6, 8, 10):
        nc = (p + 1) * (p + 2) * (p + 3) // 6
        dev = "cuda"
        s3 = torch.from_numpy(rng.uniform(-0.45, 0.45, (count, 3))).to(dev)
        far = torch.from_numpy(rng.uniform(-0.45, 0.45, (count, 3)) + np.array([2.5, 0.3, -0.2])).to(dev)
        qv = torch.from_numpy(rng.uniform(-1, 1, count)).to(dev)
        C = torch.from_numpy(rng.uniform(-1, 1, (count, nc))).to(dev)
        octs = torch.from_numpy(rng.integers(0, 8, count).astype(np.int32)).to(dev)
        outc = torch.empty((count, nc), dtype=torch.float64, device=dev)
        out4 = torch.empty((count, 4), dtype=torch.float64, device=dev)
        ops = {"P2M": lambda prec: B.dafmm_op_p2m(ctx.h, p, prec, s3, qv, outc),
               "P2L": lambda prec: B.dafmm_op_p2l(ctx.h, p, prec, far, qv, outc),
               "L2P": lambda prec: B.dafmm_op_l2p(ctx.h, p, prec, C, s3, out4),
               "M2P": lambda prec: B.dafmm_op_m2p(ctx.h, p, prec, C, far, out4),
               "M2M": lambda prec: B.dafmm_op_m2m(ctx.h, p, prec, octs, C, outc),
               "L2L": lambda prec: B.dafmm_op_l2l(ctx.h, p, prec, octs, C, outc)}
        row = {}
        for name, fn in ops.items():
            r = {}
            for pname, prec in (("gpu_fp64_ns", B.DAFMM_FP64), ("gpu_fp32_ns", B.DAFMM_FP32)):
                fn(prec)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(3):
                    fn(prec)
                e1.record()
                e1.synchronize()
                r[pname] = round(e0.elapsed_time(e1) / 3 * 1e6 / count, 4)
            row[name] = r
        # the same operators by numerical DA on the GPU (FP64, one warp per instance), on the
        # first count_da instances: the paper's generated-versus-DA comparison on one device
        count_da = {2: 1 << 15, 4: 1 << 14, 6: 1 << 12, 8: 1 << 11, 10: 1 << 10}[p]
        sub = {"s3": s3[:count_da], "far": far[:count_da], "qv": qv[:count_da], "C": C[:count_da],
               "octs": octs[:count_da], "outc": outc[:count_da], "out4": out4[:count_da]}
        r0s = torch.from_numpy(rng.integers(2, 4, (count_da, 3)) * rng.choice([-1.0, 1.0], (count_da, 3))).to(dev)
        DA = B.DAFMM_FP64 | B.DAFMM_OP_NUMERICAL_DA
        da_ops = {"P2M": lambda: B.dafmm_op_p2m(ctx.h, p, DA, sub["s3"], sub["qv"], sub["outc"]),
                  "P2L": lambda: B.dafmm_op_p2l(ctx.h, p, DA, sub["far"], sub["qv"], sub["outc"]),
                  "L2P": lambda: B.dafmm_op_l2p(ctx.h, p, DA, sub["C"], sub["s3"], sub["out4"]),
                  "M2P": lambda: B.dafmm_op_m2p(ctx.h, p, DA, sub["C"], sub["far"], sub["out4"]),
                  "M2M": lambda: B.dafmm_op_m2m(ctx.h, p, DA, sub["octs"], sub["C"], sub["outc"]),
                  "L2L": lambda: B.dafmm_op_l2l(ctx.h, p, DA, sub["octs"], sub["C"], sub["outc"]),
                  "M2L": lambda: B.dafmm_op_m2l(ctx.h, p, DA, r0s, sub["C"], sub["outc"])}
        for name, fn in da_ops.items():
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            row.setdefault(name, {})["gpu_numerical_da_ns"] = round(e0.elapsed_time(e1) * 1e6 / count_da, 2)
            if "gpu_fp64_ns" in row[name]:
                row[name]["numerical_da_over_generated_fp64"] = round(
                    row[name]["gpu_numerical_da_ns"] / row[name]["gpu_fp64_ns"], 1)
        # oracle numerical DA, one call at a time
        s1, w1, M1 = rng.uniform(-0.45, 0.45, (1, 3)), rng.uniform(-0.45, 0.45, (1, 3)) + [2.5, 0.3, -0.2], rng.uniform(-1, 1, nc)
        calls = {"P2M": lambda: O.p2m(p, s1, [1.0]), "P2L": lambda: O.p2l(p, w1, [1.0]),
                 "L2P": lambda: O.l2p(p, M1, s1[0]), "M2P": lambda: O.m2p(p, M1, w1[0]),
                 "M2M": lambda: O.m2m(p, M1, [0.25, 0.25, 0.25]), "L2L": lambda: O.l2l(p, M1, [0.25, 0.25, 0.25]),
                 "M2L": lambda: O.m2l(p, M1, [2.0, 1.0, 0.0])}
        for name, fn in calls.items():
            k = 20 if p >= 8 else 100
            t0 = time.perf_counter()
            for _ in range(k):
                fn()
            row.setdefault(name, {})["oracle_da_us"] = round((time.perf_counter() - t0) / k * 1e6, 3)
        # M2L per pair inside an evaluation
        x, q = W.uniform(1 << 18, seed=40 + p)
        tr = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=W.UNIT_CUBE, uniform_depth=4)
        pairs = tr.info()["m2l_pairs"]
        phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
        B.dafmm_set_profiling(ctx.h, True)
        for pname, prec, rot in (("gpu_fp64_ns", "fp64", 0), ("gpu_fp64_rotation_ns", "fp64", 1),
                                 ("gpu_fp32_ns", "fp32", -1)):
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_ROTATION, rot)
            tr.eval(p, phi, None, precision=prec)
            tr.eval(p, phi, None, precision=prec)
            row["M2L"][pname] = round(B.dafmm_last_phase_ms(ctx.h)["m2l"] * 1e6 / pairs, 4)
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_ROTATION, -1)
        tr.free()
        m = row["M2L"]
        m["numerical_da_over_generated_fp64"] = round(m["gpu_numerical_da_ns"] / m["gpu_fp64_ns"], 1)
        m["numerical_da_over_rotation_fp64"] = round(m["gpu_numerical_da_ns"] / m["gpu_fp64_rotation_ns"], 1)
        out["p%d" % p] = row
        del s3, far, qv, C, octs, outc, out4
    return out


def bench_leaf_size(ctx):
    """Leaf size and linear scaling on the GPU, the analogue of the paper's leaf-size study
    (Fig. 1, Table 10) and linear-scaling check (Fig. 2): a 3-D Gaussian of N particles
    (q = +1), adaptive trees, FP32 mode; time of build + evaluation for each leaf size s; the
    fastest s per (N, p) and the log-log slope of the fastest time against N."""
    import torch

    from paper_2508_02626_gb300 import workloads as W
    sizes = (10_000, 100_000, 1_000_000, 4_000_000, 10_000_000)
    orders = (2, 6, 10)
    leaf = (16, 32, 64, 128, 256, 512, 1024)
    table, best = {}, {}
    for n in sizes:
        x, q = W.gaussian(n, seed=77)
        xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        for p in orders:
            res = {}
            for s_ in leaf:
                if s_ >= n or (n >= 10_000_000 and s_ < 64):  # (1e7: the leaf sizes around the optimum)
                    continue
                t = ctx.build_tree(xt, qt, uniform_depth=-1, max_leaf=s_)
                t.eval(p, phi, None, precision="fp32")  # warm: tables, expansions
                torch.cuda.synchronize()
                t.free()
                t0 = time.perf_counter()
                t = ctx.build_tree(xt, qt, uniform_depth=-1, max_leaf=s_)
                t.eval(p, phi, None, precision="fp32")
                torch.cuda.synchronize()
                res[s_] = round((time.perf_counter() - t0) * 1e3, 3)
                t.free()
            table["N%d_p%d" % (n, p)] = res
            sb = min(res, key=res.get)
            best.setdefault("p%d" % p, {})[n] = {"s": sb, "ms": res[sb]}
    slopes = {}
    for p in orders:
        bs = best["p%d" % p]
        ns = sorted(bs)
        slopes["p%d" % p] = round(float(np.polyfit(np.log(ns), np.log([bs[k]["ms"] for k in ns]), 1)[0]), 3)
    return {"workload": "3-D Gaussian (unit sigma), q = +1, adaptive, FP32, build + eval wall time (ms)",
            "times_ms": table, "fastest": best, "loglog_slope_of_fastest": slopes}


# the paper's figures on its own workload (1M-point unit Gaussian, q = +1; i5-14600, FP64):
# Table 9 (error against the exact potential by order) and Table 11 (SDA-FMM rows: order, s,
# sigma, T in seconds), quoted as context
PAPER_TABLE9 = {2: 7.94e-4, 4: 6.30e-5, 6: 3.76e-6, 8: 1.58e-7, 10: 2.95e-8}
PAPER_TABLE11 = {3: (64, 3.12e-4, 4.70), 4: (128, 7.03e-5, 6.14), 7: (256, 8.49e-7, 20.86)}
# leaf size by order on 1M particles: Table 10's optimum (odd orders: the table of Table 11,
# else the next lower even order's)
PAPER_LEAF = {2: 64, 3: 64, 4: 128, 5: 128, 6: 256, 7: 256, 8: 256, 9: 256, 10: 512}


def bench_paper_shape(ctx, n=1_000_000, targets=5000):
    """The paper's own test (Sec. 3.5): N = 1e6 particles from a 3-D Gaussian with unit
    standard deviation, q = +1, adaptive trees with the leaf size of its Table 10.  For p = 2..10
    the relative RMS error sigma (Eq. 8) of the FP64 and FP32 modes against the exact potential
    (the oracle's direct sum, Eq. 1, on `targets` seeded particles) beside Table 9, and build +
    evaluation wall time; Table 11's SDA-FMM rows (p = 3, 4, 7 at s = 64, 128, 256) beside
    the paper's times (an i5-14600 CPU: context, not a target)."""
    import torch

    import oracle as O
    from paper_2508_02626_gb300 import workloads as W
    x, q = W.gaussian(n, seed=394)
    tg = np.sort(np.random.default_rng(395).choice(n, targets, replace=False))
    d_phi, _ = O.direct(x, q, targets=tg)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    phi = torch.empty(n, dtype=torch.float64, device="cuda")

    def sigma(a):
        return float(np.sqrt(((a[tg] - d_phi) ** 2).sum() / (d_phi ** 2).sum()))

    def solve(p, s_, prec):
        t = ctx.build_tree(xt, qt, uniform_depth=-1, max_leaf=s_)
        t.eval(p, phi, None, precision=prec)  # warm: tables, expansions
        torch.cuda.synchronize()
        t.free()
        t0 = time.perf_counter()
        t = ctx.build_tree(xt, qt, uniform_depth=-1, max_leaf=s_)
        t.eval(p, phi, None, precision=prec)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        t.free()
        return sigma(phi.cpu().numpy()), ms

    by_order = {}
    for p in range(2, 11):
        s_ = PAPER_LEAF[p]
        e64, t64 = solve(p, s_, "fp64")
        e32, t32 = solve(p, s_, "fp32")
        row = {"s": s_, "sigma_fp64": e64, "sigma_fp32": e32, "ms_fp64": round(t64, 3), "ms_fp32": round(t32, 3)}
        if p in PAPER_TABLE9:
            row["paper_sigma"] = PAPER_TABLE9[p]
        by_order["p%d" % p] = row
    t11 = {}
    for p, (s_, sig, sec) in PAPER_TABLE11.items():
        r = by_order["p%d" % p]
        t11["p%d_s%d" % (p, s_)] = {"sigma_fp64": r["sigma_fp64"], "ms_fp64": r["ms_fp64"],
                                    "sigma_fp32": r["sigma_fp32"], "ms_fp32": r["ms_fp32"],
                                    "paper_sigma": sig, "paper_seconds_i5_14600": sec}
    return {"workload": "3-D Gaussian (unit sigma), N=%d, q=+1, adaptive, leaf size of Table 10; sigma (Eq. 8) "
                        "against the direct sum on %d seeded particles; time = build + eval wall" % (n, targets),
            "by_order": by_order, "table11": t11}


def cpu_baseline(x, q, dom, cfg, phi_gpu, E_gpu, phi_by_order=None, mode_results=None):
    """The oracle FMM (plain C, all host cores) timed on one full solve of the workload: same
    tree and order, every particle a target, nothing extrapolated (about 15 s on 16 Arm cores,
    23 s on 8 x86 cores).  Its result also gives the GPU's error against the oracle over all
    particles (relative L2, and the worst single target relative to max(|value|, median
    |value|)); 2000 seeded random particles give the errors of both against the direct sum
    (Eq. 1), for the potential and the field."""
    import oracle as O

    n, p, depth = cfg["n"], cfg["order"], cfg["uniform_depth"]
    cores = O.default_threads()
    t0 = time.perf_counter()
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=depth, nthreads=cores)
    t_full = time.perf_counter() - t0
    td = np.sort(np.random.default_rng(123).choice(n, 2000, replace=False))
    d_phi, d_E = O.direct(x, q, targets=td)

    def rel(a, b):
        return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))

    def worst(a, b):
        if a.ndim == 1:
            a, b = a[:, None], b[:, None]
        m = np.linalg.norm(b, axis=1)
        return float((np.linalg.norm(a - b, axis=1) / np.maximum(m, np.median(m))).max())

    cpu = {"value": n / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "one full oracle FMM solve of all %d particles (%.1f s), nothing extrapolated" % (n, t_full)}
    acc = {"targets": int(n), "direct_sum_targets": int(len(td)),
           "rel_l2_phi_vs_oracle": rel(phi_gpu, ref_phi), "rel_l2_field_vs_oracle": rel(E_gpu, ref_E),
           "worst_target_phi_vs_oracle": worst(phi_gpu, ref_phi), "worst_target_field_vs_oracle": worst(E_gpu, ref_E),
           "rel_l2_phi_vs_direct": rel(phi_gpu[td], d_phi),
           "oracle_rel_l2_phi_vs_direct": rel(ref_phi[td], d_phi),
           "rel_l2_field_vs_direct": rel(E_gpu[td], d_E),
           "oracle_rel_l2_field_vs_direct": rel(ref_E[td], d_E)}
    if mode_results:  # the other precision modes on the same tree, against the same oracle solve
        acc["modes"] = {m: {"rel_l2_phi_vs_oracle": rel(ph, ref_phi), "rel_l2_field_vs_oracle": rel(Ef, ref_E)}
                        for m, (ph, Ef) in mode_results.items()}
    if phi_by_order:
        by = {"p%d" % po: rel(ph[td], d_phi) for po, ph in sorted(phi_by_order.items())}
        reach = [po for po, ph in sorted(phi_by_order.items()) if rel(ph[td], d_phi) <= 1e-7]
        acc["fp64_rel_l2_phi_vs_direct_by_order"] = by
        acc["smallest_order_reaching_1e-7"] = reach[0] if reach else None
    return cpu, acc


def run_reference(args, rank, world):
    """CPU oracle arm: every step, warm-up steps included, is one full oracle FMM solve of the
    workload (all particles, all host cores); the rate is particles over the mean step time."""
    import oracle as O
    from paper_2508_02626_gb300 import workloads as W

    cfg = W.C2
    x, q, dom = W.make(cfg)
    n, p, depth = cfg["n"], cfg["order"], cfg["uniform_depth"]
    cores = O.default_threads()

    def step():
        t0 = time.perf_counter()
        O.fmm(x, q, dom, p, uniform_depth=depth, nthreads=cores)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    t_step = float(np.mean(ts))
    value = n / t_step
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded uniform, PCG64 seed 2002)",
            "config": {"workload": "uniform N=1e6, q~U[-1,1], octree depth 5, order p=8, theta=1",
                       "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: one full oracle FMM solve of all %d particles, nothing "
                                       "extrapolated" % n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--no-modes", action="store_true", help="skip the MIXED / FP64 comparison runs")
    ap.add_argument("--modes", default="", help="comparison modes to run (comma-separated; default all): "
                                                "mixed, fp64, fp64_dense_m2l, fp32_tf32_m2l, ff")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the unit-rate probes (dafmm_probe_peak)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the adaptive, batched and serving workloads (N = 1 only)")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--adaptive-n", type=int, default=0, help="particles of the adaptive workload (0: 4e6)")
    ap.add_argument("--adaptive-modes", default="mixed,fp32", help="precision modes of the adaptive workload")
    ap.add_argument("--sections", default="adaptive,batch,serving,operators,leafsize,paper",
                    help="comma-separated extra workloads at N = 1: adaptive, batch, serving, operators, leafsize, "
                         "paper")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
