"""Throughput of the randomized von Neumann entropy estimators on GB300.

Default workload (one step = one density matrix through the whole hot path):
dense n = 8192 density matrix R = Psi diag(p) Psi^T (Psi from the QR of a
seeded Gaussian matrix, p_i ~ i^-1.5 on the top 2048 states and a 1e-9 floor
on the rest, unit trace, FP64 in HBM).  Per step: bf16 hi/lo split of R,
30 power-method products (Algorithm alg:power) -> u, then the Chebyshev
(Algorithm 1b, m = 40) and Taylor (Algorithm 1a, m = 40) recurrences on
s = 128 Gaussian probes sharing every pass over R (41 tensor-core steps),
FP64 combine, and the estimates copied back to the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|bf16x3|f64]
                    [--workload dense_powerlaw_n8192|dense_exp_n512|band33_n1e7|
                                lowrank_n8192_k64|krylov_n8192_b64|learned_n8192|batched256|
                                hermitian_n5000]
                    [--impl reference]

Prints one JSON line.  `--impl reference` times the CPU FP64 oracle on the
host cores on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


def profiled_traffic(profile_name, source):
    """DRAM bytes per launch recorded in profiles/<profile_name> by an ncu
    capture, or None when the kernel source changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", profile_name)
    src = os.path.join(ROOT, "paper_1801_01072_gb300", "csrc", source)
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    text = open(prof).read()
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if f"{source} {digest}" not in text:
        return None
    for line in text.splitlines():
        if line.strip().startswith("- traffic_bytes_per_launch:"):
            return int(line.split(":")[1].split()[0])
    return None


def peak_value(d, *keys):
    for k in keys:
        v = d.get(k)
        if isinstance(v, (int, float)):
            return float(v)
        if isinstance(v, dict):
            for kk in ("value", "median", "mean"):
                if isinstance(v.get(kk), (int, float)):
                    return float(v[kk])
    return None


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def make_workload(name):
    w = dict(synth.WORKLOADS[name])
    if w["kind"] == "hermitian":
        return w, None, synth.spectrum_exponential(w["n"], w["tau"])
    if w["kind"] == "batched":
        return w, synth.batched_specs(w["count"], w["seed"], w["n_lo"], w["n_hi"]), None
    if w["kind"] == "learned":
        R, p, _ = synth.dense_powerlaw(w["n"], w["k"], w["alpha"], w["floor"], w["seed"])
        return w, R, p
    if w["kind"] == "lowrank":
        R, p, _ = synth.dense_lowrank(w["n"], w["k"], w["tau"], w["seed"])
        return w, R, p
    if w["kind"] == "dense":
        if w["spectrum"] == "powerlaw":
            R, p, _ = synth.dense_powerlaw(w["n"], w["k"], w["alpha"], w["floor"], w["seed"])
        else:
            R, p, _ = synth.dense_exp(w["n"], w["tau"], w["seed"])
        return w, R, p
    vals = synth.band_diag_dominant(w["n"], w["half_bw"], w["offdiag_scale"], w["seed"],
                                    dtype=np.float32)
    return w, vals, None


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class Clocks:
    """SM clocks and clock-event reasons sampled during the timed region:
    NVML queries (read-only) every 5 ms from a helper thread, matched to the
    CUDA device by PCI bus id; nvidia-smi at 200 ms when NVML is missing."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_slowdown"}

    def __init__(self, device_index=0, period_s=0.005):
        self.p = None
        self.th = None
        self.nv = None
        self.samples = []
        self.period = period_s
        self.path = os.path.join(tempfile.gettempdir(), f"vne_clocks_{os.getpid()}.csv")
        self.dev = device_index

    def _nvml(self):
        import ctypes as C
        try:
            lib = C.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = C.c_void_p()
            ok = False
            try:
                import torch
                pr = torch.cuda.get_device_properties(self.dev)
                bus = "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), C.byref(h)) == 0
            except Exception:
                ok = False
            if not ok and lib.nvmlDeviceGetHandleByIndex_v2(self.dev, C.byref(h)) != 0:
                return None
            rs = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            return lib, h, rs
        except Exception:
            return None

    def _loop(self):
        import ctypes as C
        lib, h, rs = self.nv
        clk, mx, why = C.c_uint(), C.c_uint(), C.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) == 0 and
                    rs(h, C.byref(why)) == 0):
                self.samples.append((clk.value, mx.value, why.value))
            self.stop.wait(self.period)

    def __enter__(self):
        import threading
        self.nv = self._nvml()
        if self.nv is not None:
            self.stop = threading.Event()
            self.th = threading.Thread(target=self._loop, daemon=True)
            self.th.start()
            return self
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}",
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.th is not None:
            self.stop.set()
            self.th.join(timeout=5)
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        if self.th is not None:
            for c, m, w in self.samples:
                sm.append(float(c))
                mx.append(float(m))
                for bit, nm in self.REASONS.items():
                    if w & bit:
                        reasons.add(nm)
            src = f"NVML every {self.period * 1e3:.0f} ms"
        else:
            if self.p is None or not os.path.exists(self.path):
                return None
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1].split()[0]))
                    mx.append(float(parts[2].split()[0]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            src = "nvidia-smi every 200 ms"
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm), "source": src}


# --------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# --------------------------------------------------------------------------

def oracle_sample_time(w, R, s_sample):
    """Time the oracle on the full matrix with s_sample of the s probes:
    power method + both recurrences.  Returns (seconds extrapolated to the
    full s, description, threads)."""
    import oracle as O
    from oracle import rng

    n, m, s = w["n"], w["m"], w["s"]
    if w["kind"] == "band":
        Rop = O.Dia(R)
    else:
        Rop = R
    t0 = time.perf_counter()
    lam, _ = O.power_method(Rop, rng.power_start(n, 1, w["seed"]), w["power_iters"])
    t1 = time.perf_counter()
    u = O.interval_u(lam, 1.0)
    G = rng.probes(n, s, w["seed"], w["probe"])[:, :s_sample]
    O.chebyshev_moments(Rop, G, u, m)
    if w["kind"] == "dense":
        O.taylor_terms(Rop, G, u, m)
    if w["kind"] == "dense_cheb":
        import oracle.learned as OL
        theta = synth.mlp_init(1)
        OL.forward(theta, np.zeros((1, OL.N_IN)))
    t2 = time.perf_counter()
    full = (t1 - t0) + (t2 - t1) * (s / s_sample)
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count() or 1
    est = {"dense": "Chebyshev + Taylor", "dense_cheb": "Chebyshev + network forward"}.get(
        w["kind"], "Chebyshev")
    desc = (f"oracle (NumPy FP64) on the full n={n} matrix: {w['power_iters']} power-method "
            f"products + {est} recurrences, m={m}, on {s_sample} of the s={s} probes, "
            f"time scaled by s/{s_sample} for the recurrence part")
    return full, desc, threads


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def oracle_full_time(w, R):
    """Time one whole oracle estimate of a dense workload: the power method
    (t products), u, all s probes, and the Chebyshev and Taylor recurrences
    (or Chebyshev alone).  Nothing is sampled or scaled.  Returns (seconds,
    description, threads)."""
    import oracle as O
    from oracle import rng

    n, m, s = w["n"], w["m"], w["s"]
    t0 = time.perf_counter()
    lam, _ = O.power_method(R, rng.power_start(n, 1, w["seed"]), w["power_iters"])
    u = O.interval_u(lam, 1.0)
    G = rng.probes(n, s, w["seed"], w["probe"])
    O.chebyshev_estimate_from_moments(O.chebyshev_moments(R, G, u, m), u)
    both = w["kind"] == "dense"
    if both:
        O.taylor_estimate_from_terms(O.taylor_terms(R, G, u, m), u)
    if w["kind"] == "dense_cheb":  # the learned form: plus the network's forward pass
        import oracle.learned as OL
        OL.forward(synth.mlp_init(1), np.zeros((1, OL.N_IN)))
    t = time.perf_counter() - t0
    desc = (f"oracle (NumPy FP64) whole estimate on the full n={n} matrix: {w['power_iters']} "
            f"power-method products, all s={s} {w['probe']} probes, "
            f"{'Chebyshev + Taylor' if both else 'Chebyshev'} m={m}; timed, not scaled")
    return t, desc, blas_threads()


def oracle_projection_time(w, R):
    """Time one oracle call of Algorithm alg:EN on the full matrix."""
    import oracle.projection as OP

    t0 = time.perf_counter()
    if w.get("krylov", 0):
        OP.estimate_block_krylov(R, w["k"], w["s"], w["krylov"], w["sketch"], seed=w["seed"])
    else:
        OP.estimate_projection(R, w["k"], w["s"], w["sketch"], seed=w["seed"])
    t = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count() or 1
    desc = (f"oracle (NumPy FP64) Algorithm EN on the full n={w['n']} rank-{w['k']} matrix: "
            f"{w['sketch']} sketch s={w['s']}, R Pi and its SVD, one whole estimate"
            if not w.get("krylov", 0) else
            f"oracle (NumPy FP64) block Krylov on the full n={w['n']} rank-{w['k']} matrix: "
            f"block {w['s']}, {w['krylov']} iterations, one whole estimate")
    return t, desc, threads


PROJ_METRIC = ("entropies/s (rank-64 n=8192 density matrices through Algorithm EN: Gaussian "
               "sketch s=256, R Pi, singular values, top-64 entropy)")


KRYLOV_METRIC = ("entropies/s (rank-64 n=8192 density matrices through the block-Krylov "
                 "projection: Gaussian block 64, 4 iterations, top-64 Ritz values + tail)")


def run_gpu_projection(args, w, Rh, p, world, rank, local, dev):
    import torch
    import torch.distributed as dist

    import paper_1801_01072_gb300 as vne

    n, k, s = w["n"], w["k"], w["s"]
    # R Pi on the tensor cores (bf16x3) unless a CUDA-core precision is asked for
    prec = args.precision if args.precision in ("f32", "f64", "bf16x3", "bf16x6") else "bf16x3"
    tc = prec.startswith("bf16")
    Rd = torch.as_tensor(Rh).to(dev)
    seed = w["seed"] + 1000 * rank

    q = w.get("krylov", 0)

    def step(R):
        return vne.entropy_projection(R, k, s, w["sketch"], seed=seed, precision=prec,
                                      krylov_iters=q)

    h = vne._handle(local)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        out = step(Rd)
    torch.cuda.synchronize()
    h.profile(True)
    n_launch0 = h.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            out = step(Rd)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    n_launch = h.launch_count() - n_launch0
    ms = ev0.elapsed_time(ev1)
    k_ms, k_n = h.profile_read(0 if tc else 1)
    h.profile(False)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())

    Rpin = torch.as_tensor(Rh).pin_memory()
    step(Rpin)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 4)
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(Rpin)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - e0) / e2e_steps * 1e3

    rel = None
    if rank == 0 and prec != "f64" and not args.skip_f64_check:
        ref = vne.entropy_projection(Rd, k, s, w["sketch"], seed=seed, precision="f64",
                                     krylov_iters=q)
        rel = {"H": abs(out.H - ref.H) / abs(ref.H),
               "p_max_rel_to_p1": float(np.abs(out.p - ref.p).max() / ref.p[0])}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk, pk_src = peaks()
    # the products R X: 2 n^2 s algorithmic flops per product (q + 1 products).
    # Tensor cores (bf16x3 / bf16x6): against the measured BF16 burst peak (the
    # split modes issue 3 / 6 MMAs per algorithmic product, reported beside);
    # CUDA cores: FP32 152 SMs x 128 lanes x 2 flops x 2.07 GHz, FP64 nominal.
    flops = 2.0 * n * n * s * (q + 1) * args.steps
    achieved = flops / (k_ms / 1e3) / 1e12 if k_ms > 0 else None
    if tc:
        peak = peak_value(pk, "bf16_tflops", "bf16_tflops_sustained")
        mma = {"bf16x3": 3, "bf16x6": 6}[prec]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if (achieved and peak) else None, "traffic": None,
                "kernel": "k_tc_step (plain product)", "launches": k_n,
                "avg_launch_us": k_ms / max(k_n, 1) * 1e3,
                "mma_tflops_issued": achieved * mma if achieved else None,
                "peak_source": pk_src + " bf16 burst"}
    else:
        peak = 152 * 128 * 2 * 2.07e9 / 1e12 if prec == "f32" else 1.25
        traffic = profiled_traffic("k_simt_step_f32_lowrank_n8192_k64.md", "vne_dense_simt.cu") \
            if (prec == "f32" and args.workload == "lowrank_n8192_k64") else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": "k_simt_step", "launches": k_n, "avg_launch_us": k_ms / max(k_n, 1) * 1e3,
                "peak_source": "derived: FP32 lanes x 2 x max SM clock" if prec == "f32"
                else "nominal FP64"}
    cpu = None
    if world == 1 and not args.skip_cpu:
        t_cpu, desc, threads = oracle_projection_time(w, Rh)
        cpu = {"value": 1.0 / t_cpu, "unit": "entropies/s", "cores": threads, "kind": "oracle",
               "sample": desc}
    line = {
        "metric": PROJ_METRIC if not q else KRYLOV_METRIC,
        "value": world * args.steps / (ms_max / 1e3),
        "unit": "entropies/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": prec,
        "data": "synthetic (seeded rank-k density matrices, no dataset)",
        "config": {"workload": args.workload, "n": n, "k": k, "s": s, "sketch": w["sketch"],
                   "krylov_iters": q, "precision": prec, "input": "R FP64 resident in HBM",
                   "l2": "inputs larger than L2 (R is %.0f MB)" % (Rh.nbytes / 1e6),
                   "parallelism": f"independent matrices, {world} GPU(s)"},
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "entropies/s",
                "h2d_bytes_per_step": int(Rh.nbytes), "d2h_bytes_per_step": (k + 1) * 8},
        "gpu_launches": int(n_launch),
        "phases_ms_per_step": {"product": k_ms / args.steps,
                               "other": ms_max / args.steps - k_ms / args.steps},
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "rel_err_vs_f64": rel,
        "estimates": {"H": out.H, "H_exact": float(-(p * np.log(p)).sum())},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


LEARNED_METRIC = ("entropies/s (n=8192 density matrices through power method + Chebyshev m=16 "
                  "on BF16 tensor cores, s=128 Gaussian probes, + learned correction)")


def run_gpu_learned(args, w, Rh, p, world, rank, local, dev):
    import torch
    import torch.distributed as dist

    import paper_1801_01072_gb300 as vne
    from paper_1801_01072_gb300 import learned

    n, m, s = w["n"], w["m"], w["s"]
    prec = args.precision if args.precision in ("bf16", "bf16x3", "f64", "f32") else "bf16"
    Rd = torch.as_tensor(Rh).to(dev)
    seed = w["seed"] + 1000 * rank
    H_exact = float(-(p[p > 0] * np.log(p[p > 0])).sum())
    # training (outside the timed region): sampled spectra, the library's kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    data = learned.spectral_samples(synth.learned_sample_params(w["train_count"], 1), s=s,
                                    device=local)
    theta0 = torch.tensor(synth.mlp_init(1), dtype=torch.float32).to(dev)
    theta, hist = learned.train(theta0, data["features"], data["target"],
                                epochs=w["train_epochs"], batch=1024, lr=2e-3, report_every=1000)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del data
    # held out: 10k sampled spectra at n = 8192 (outside the training sizes),
    # degree 16 + network against plain degree 16 and plain degree 64 on the
    # same probes, errors against the exact entropies
    held = {}
    sp = synth.learned_sample_params(10000, 77, 8192, 8192)
    a16 = learned.spectral_samples(sp, m=16, s=s, device=local)
    a64 = learned.spectral_samples(sp, m=64, s=s, device=local)
    corr = learned.mlp_forward(theta, a16["features"]).double()
    nn_ = torch.tensor(sp["n"], dtype=torch.float64, device=dev)
    uu = torch.exp(10.0 * a16["features"][:, 18].double())
    He = a16["H_exact"]
    for key, est in (("degree16", a16["H_low"]), ("degree64", a64["H_low"]),
                     ("degree16_plus_network", a16["H_low"] + corr * nn_ * uu / 100.0)):
        r = ((est - He).abs() / He)
        held[key] = {"mean_rel_err": float(r.mean()), "p90_rel_err": float(r.quantile(0.9))}
    del a16, a64

    def step(R):
        return learned.entropy_chebyshev_learned(R, theta, s=s, seed=seed, precision=prec,
                                                 power_iters=w["power_iters"])

    h = vne._handle(local)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        out = step(Rd)
    torch.cuda.synchronize()
    h.profile(True)
    n_launch0 = h.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            out = step(Rd)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    n_launch = h.launch_count() - n_launch0
    ms = ev0.elapsed_time(ev1)
    k_ms, k_n = h.profile_read(0 if prec in ("bf16", "bf16x3") else 1)
    h.profile(False)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    Rpin = torch.as_tensor(Rh).pin_memory()
    step(Rpin)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 4)
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(Rpin)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - e0) / e2e_steps * 1e3
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    # the plain full-degree estimator on the same GPU: FP64, degree m_ref
    torch.cuda.synchronize()
    f0 = time.perf_counter()
    ref = vne.entropy_chebyshev(Rd, w["m_ref"], s, seed=seed, probe="gaussian", precision="f64",
                                power_iters=w["power_iters"], u_scale=1.05)
    torch.cuda.synchronize()
    f64_ms = (time.perf_counter() - f0) * 1e3
    pk, pk_src = peaks()
    flops = 2.0 * n * n * s * m * args.steps
    achieved = flops / (k_ms / 1e3) / 1e12 if k_ms > 0 else None
    peak = peak_value(pk, "bf16_tflops", "bf16_tflops_sustained") if prec.startswith("bf16") else None
    roof = {"bound": "tensor" if peak else "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if (achieved and peak) else None,
            "traffic": None, "kernel": "k_tc_step" if peak else "k_simt_step", "launches": k_n,
            "avg_launch_us": k_ms / max(k_n, 1) * 1e3,
            "peak_source": pk_src + (" bf16 burst" if peak else "")}
    cpu = None
    if world == 1 and not args.skip_cpu:
        t_cpu, desc, threads = oracle_full_time(dict(w, kind="dense_cheb"), Rh)
        cpu = {"value": 1.0 / t_cpu, "unit": "entropies/s", "cores": threads, "kind": "oracle",
               "sample": desc}
    value = world * args.steps / (ms_max / 1e3)
    line = {
        "metric": LEARNED_METRIC, "value": value, "unit": "entropies/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
        "data": "synthetic (seeded density matrix and sampled training spectra, no dataset)",
        "config": {"workload": args.workload, "n": n, "m": m, "s": s, "probe": "gaussian",
                   "power_iters": w["power_iters"], "precision": prec, "u_scale": 1.05,
                   "input": "R FP64 resident in HBM",
                   "l2": "inputs larger than L2 (R is %.0f MB)" % (Rh.nbytes / 1e6),
                   "parallelism": f"independent matrices, {world} GPU(s)"},
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "entropies/s",
                "h2d_bytes_per_step": int(Rh.nbytes), "d2h_bytes_per_step": 200 * 8},
        "gpu_launches": int(n_launch),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "training": {"spectra": w["train_count"], "epochs": w["train_epochs"],
                     "seconds_incl_sampling": train_s, "final_loss": hist[-1][1] if hist else None},
        "held_out_10k_spectra_n8192": held,
        "vs_plain_fp64": {"m": w["m_ref"], "ms": f64_ms, "speedup": f64_ms / (ms_max / args.steps),
                          "rel_err_exact_plain_fp64": abs(ref.H - H_exact) / H_exact},
        "estimates": {"H_learned": out.H, "H_plain_m16": out.H_plain, "H_exact": H_exact,
                      "rel_err_exact_learned": abs(out.H - H_exact) / H_exact,
                      "rel_err_exact_plain_m16": abs(out.H_plain - H_exact) / H_exact,
                      "u": out.u},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


BATCH_METRIC = ("entropies/s (256 dense density matrices, n log-uniform in [256, 4096], "
                "power method + Chebyshev m=24 on BF16 tensor cores, s=32, one batched call)")


def batch_matrices(specs, dev):
    """R_b = Q diag(p) Q^T with Q the (sign-fixed) QR factor of a seeded
    Gaussian matrix, built on the GPU (FP32 QR, FP64 result)."""
    import torch

    mats = []
    for n, p, seed in specs:
        g = torch.Generator(device=dev).manual_seed(seed)
        A = torch.randn(n, n, generator=g, device=dev, dtype=torch.float32)
        Q, Rr = torch.linalg.qr(A)
        Q = (Q * torch.sign(torch.diagonal(Rr))[None, :]).double()
        R = (Q * torch.tensor(p, device=dev)[None, :]) @ Q.T
        mats.append((0.5 * (R + R.T)).contiguous())
    return mats


def run_gpu_batched(args, w, specs, world, rank, local, dev):
    import torch
    import torch.distributed as dist

    import paper_1801_01072_gb300 as vne

    m, s = w["m"], w["s"]
    prec = args.precision if args.precision in ("bf16", "bf16x3", "f64", "f32") else "bf16"
    seed = w["seed"] + 1000 * rank
    t0 = time.perf_counter()
    mats = batch_matrices(specs, dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    # autotune the tensor-core tile per size bucket (the largest matrix of each)
    tuned = {}
    if prec.startswith("bf16"):
        buckets = {}
        for i, (n, _, _) in enumerate(specs):
            b = int(np.ceil(np.log2(max(1, -(-n // 128)))))
            if b not in buckets or n > specs[buckets[b]][0]:
                buckets[b] = i
        for b, i in sorted(buckets.items()):
            shape, us = vne.autotune(mats[i], m, s, precision=prec, method="chebyshev",
                                     seed=seed, probe=w["probe"], power_iters=w["power_iters"])
            tuned[str(specs[i][0])] = {"shape": list(shape), "us_per_step": us}

    def step():
        return vne.entropy_batched(mats, m, s, seed=seed, probe=w["probe"], precision=prec,
                                   method="chebyshev", use_graph=True,
                                   power_iters=w["power_iters"])

    stream = torch.cuda.current_stream(dev)
    h = vne._handle(local)
    c0 = h.launch_count()
    out = step()  # captures the graph: counts the kernels of one batch
    per_batch = h.launch_count() - c0
    for _ in range(args.warmup - 1):
        out = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            out = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    # the same matrices one call at a time (no batching, no graph)
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    single = [vne.entropy_chebyshev(R, m, s, seed=seed, probe=w["probe"], precision=prec,
                                    power_iters=w["power_iters"]).H for R in mats]
    torch.cuda.synchronize()
    single_ms = (time.perf_counter() - s0) * 1e3
    # the same batch on the stream path (per-matrix step launches on 32 streams
    # in one graph, no persistent recurrence), for comparison
    os.environ["VNE_BATCH_PERSISTENT"] = "0"
    for _ in range(2):
        out_streams = step()
    torch.cuda.synchronize()
    s1 = time.perf_counter()
    for _ in range(3):
        out_streams = step()
    torch.cuda.synchronize()
    streams_ms = (time.perf_counter() - s1) / 3 * 1e3
    del os.environ["VNE_BATCH_PERSISTENT"]
    # end to end: the matrices copied from pinned host memory inside the step
    host = [R.cpu().pin_memory() for R in mats]
    h2d = int(sum(x.numel() * 8 for x in host))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(2):
        for dst, src in zip(mats, host):
            dst.copy_(src, non_blocking=True)
        step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - e0) / 2 * 1e3
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    H_exact = np.array([float(-(p * np.log(p)).sum()) for _, p, _ in specs])
    rel = np.abs(out[0] - H_exact) / H_exact
    # s = 32 columns per pass over R: every kernel of the batch streams R, so
    # the bound is HBM.  Algorithmic bytes per matrix: the FP64 input read once
    # (8 n^2) and its bf16 copy written (2 n^2), then one bf16 read of R per
    # power-method product (t + 1) and per recurrence step (m): 2 n^2 each.
    bytes_alg = sum((10.0 + 2.0 * (w["power_iters"] + 1 + m)) * n * n for n, _, _ in specs)
    flops = sum(2.0 * n * n * s * m for n, _, _ in specs)
    pk, pk_src = peaks()
    step_s = ms_max / args.steps / 1e3
    achieved = bytes_alg / step_s / 1e9
    peak = peak_value(pk, "hbm_gbs")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if peak else None, "traffic": None,
            "kernel": "whole batch (all kernels of the step under one graph launch)",
            "algorithmic_bytes_per_step": bytes_alg,
            "recurrence_tflops": flops / step_s / 1e12, "peak_source": pk_src + " hbm"}
    cpu = None
    if world == 1 and not args.skip_cpu:
        import oracle as O
        from oracle import rng
        idx = list(range(0, len(specs), max(1, len(specs) // 4)))[:4]
        c0 = time.perf_counter()
        tot_full = 0.0
        for i in idx:
            n, p, sd = specs[i]
            R = mats[i].cpu().numpy()
            lam, _ = O.power_method(R, rng.power_start(n, 1, seed), w["power_iters"])
            ta = time.perf_counter()
            G = rng.probes(n, s, seed, w["probe"])[:, :4]
            O.chebyshev_moments(R, G, O.interval_u(lam, 1.0), m)
            tb = time.perf_counter()
            tot_full += (ta - c0) + (tb - ta) * s / 4
            c0 = time.perf_counter()
        per = tot_full / len(idx)
        try:
            from threadpoolctl import threadpool_info
            threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
        except Exception:
            threads = os.cpu_count() or 1
        cpu = {"value": 1.0 / per, "unit": "entropies/s", "cores": threads, "kind": "oracle",
               "sample": f"oracle (NumPy FP64) on {len(idx)} of the {len(specs)} matrices: power "
                         f"method + Chebyshev m={m} on 4 of the s={s} probes, recurrence time "
                         f"scaled by s/4, mean per matrix"}
    line = {
        "metric": BATCH_METRIC, "value": world * len(specs) * args.steps / (ms_max / 1e3),
        "unit": "entropies/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec,
        "data": "synthetic (seeded uneven density matrices built on the GPU, no dataset)",
        "config": {"workload": args.workload, "count": len(specs), "n_range": [w["n_lo"], w["n_hi"]],
                   "n_total": int(sum(n for n, _, _ in specs)), "m": m, "s": s,
                   "probe": w["probe"], "power_iters": w["power_iters"], "precision": prec,
                   "input": "FP64 matrices resident in HBM (%.1f GB)" % (h2d / 1e9),
                   "l2": "inputs larger than L2", "graph": "one CUDA graph launch per step",
                   "parallelism": f"prologues on 32 streams, every recurrence step of the batch "
                                  f"in one persistent launch, inside one graph; {world} GPU(s)"},
        "e2e": {"value": world * len(specs) * 1e3 / e2e_ms, "unit": "entropies/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(specs) * 200 * 8},
        "gpu_launches": int(per_batch * args.steps),  # kernels of the replayed graph
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "vs_single_calls": {"ms": single_ms, "speedup": single_ms / (ms_max / args.steps)},
        "vs_stream_path": {"ms": streams_ms, "speedup": streams_ms / (ms_max / args.steps)},
        "autotuned": tuned,
        "matrix_generation_s": gen_s,
        "estimates": {"rel_err_exact_mean": float(rel.mean()), "rel_err_exact_max": float(rel.max()),
                      "max_rel_diff_vs_single_calls": float(
                          np.max(np.abs(out[0] - np.array(single)) / np.abs(np.array(single)))),
                      "max_rel_diff_vs_stream_path": float(
                          np.max(np.abs(out[0] - out_streams[0]) / np.abs(out_streams[0])))},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


HERM_METRIC = ("entropies/s (5000 x 5000 complex Hermitian density matrices, power method + "
               "Algorithms alg1a_complex + alg1b_complex, m=10, s=100, BF16 tensor cores)")


def hermitian_matrix(w, dev):
    """R = U diag(p) U^H with U the (phase-fixed) QR factor of a seeded complex
    Gaussian matrix, built on the GPU (complex64 QR, complex128 result)."""
    import torch

    n = w["n"]
    p = synth.spectrum_exponential(n, w["tau"])
    g = torch.Generator(device=dev).manual_seed(w["seed"])
    A = torch.complex(torch.randn(n, n, generator=g, device=dev),
                      torch.randn(n, n, generator=g, device=dev))
    Q, Rr = torch.linalg.qr(A)
    d = torch.diagonal(Rr)
    Q = (Q * (d / d.abs())[None, :]).to(torch.complex128)
    R = (Q * torch.tensor(p, device=dev, dtype=torch.float64)[None, :]) @ Q.conj().T
    return (0.5 * (R + R.conj().T)).contiguous(), p


def run_gpu_hermitian(args, w, p, world, rank, local, dev):
    import torch
    import torch.distributed as dist

    import paper_1801_01072_gb300 as vne

    n, m, s = w["n"], w["m"], w["s"]
    prec = args.precision if args.precision in ("bf16", "bf16x3", "f64", "f32") else "bf16"
    Rd, p = hermitian_matrix(w, dev)
    seed = w["seed"] + 1000 * rank

    def step(R):
        # u from the power method on the same matrix (the experiments of
        # Section 6 vary u; the printed bound u = 1 is far too loose here)
        lam = vne.lambda_max(R, power_iters=30, precision=prec)
        return vne.entropy_both(R, m, s, seed=seed, probe="gaussian", precision=prec, u=lam)

    h = vne._handle(local)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        out = step(Rd)
    torch.cuda.synchronize()
    h.profile(True)
    n_launch0 = h.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            out = step(Rd)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    n_launch = h.launch_count() - n_launch0
    ms = ev0.elapsed_time(ev1)
    tc = prec.startswith("bf16")
    k_ms, k_n = h.profile_read(0 if tc else 1)
    h.profile(False)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    Rpin = Rd.cpu().pin_memory()
    step(Rpin)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 4)
    for _ in range(e2e_steps):
        step(Rpin)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - e0) / e2e_steps * 1e3
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    rel = None
    if prec != "f64" and not args.skip_f64_check:
        lam = vne.lambda_max(Rd, power_iters=30, precision="f64")
        ref = vne.entropy_both(Rd, m, s, seed=seed, probe="gaussian", precision="f64", u=lam)
        rel = {"chebyshev": abs(out.H_chebyshev - ref.H_chebyshev) / abs(ref.H_chebyshev),
               "taylor": abs(out.H_taylor - ref.H_taylor) / abs(ref.H_taylor)}
    H_exact = float(-(p * np.log(p)).sum())
    pk, pk_src = peaks()
    # the embedding is 2n x 2n: 2 (2n)^2 flops per probe column and step
    cols = 2 * s * m + s
    flops = 2.0 * (2 * n) ** 2 * cols * args.steps
    achieved = flops / (k_ms / 1e3) / 1e12 if k_ms > 0 else None
    peak = peak_value(pk, "bf16_tflops", "bf16_tflops_sustained") if tc else None
    roof = {"bound": "tensor" if tc else "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if (achieved and peak) else None,
            "traffic": None, "kernel": "k_tc_step" if tc else "k_simt_step", "launches": k_n,
            "avg_launch_us": k_ms / max(k_n, 1) * 1e3,
            "peak_source": pk_src + (" bf16 burst" if tc else "")}
    cpu = None
    if world == 1 and not args.skip_cpu:
        import oracle.hermitian as OH
        from oracle import rng
        Rh = Rd.cpu().numpy()
        sp = 4
        G = rng.gaussian(n, s, seed)[:, :sp]
        c0 = time.perf_counter()
        OH.chebyshev_moments_complex(Rh, G, 1.0, m)
        OH.taylor_terms_complex(Rh, G, 1.0, m)
        t_cpu = (time.perf_counter() - c0) * s / sp
        try:
            from threadpoolctl import threadpool_info
            threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
        except Exception:
            threads = os.cpu_count() or 1
        cpu = {"value": 1.0 / t_cpu, "unit": "entropies/s", "cores": threads, "kind": "oracle",
               "sample": f"oracle (NumPy complex128) Chebyshev + Taylor recurrences m={m} on "
                         f"{sp} of the s={s} probes of the full matrix, scaled by s/{sp} (the "
                         f"30 power-method products, 1.5% of the products, not included)"}
    line = {
        "metric": HERM_METRIC, "value": world * args.steps / (ms_max / 1e3),
        "unit": "entropies/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec,
        "data": "synthetic (seeded complex density matrix built on the GPU, no dataset)",
        "config": {"workload": args.workload, "n": n, "m": m, "s": s, "probe": "gaussian",
                   "u": "power method, 30 products", "precision": prec,
                   "input": "R complex128 resident in HBM (%.0f MB)"
                   % (n * n * 16 / 1e6), "l2": "inputs larger than L2",
                   "parallelism": f"independent matrices, {world} GPU(s)"},
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "entropies/s",
                "h2d_bytes_per_step": n * n * 16, "d2h_bytes_per_step": 200 * 8},
        "gpu_launches": int(n_launch),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "rel_err_vs_f64": rel,
        "estimates": {"H_chebyshev": out.H_chebyshev, "H_taylor": out.H_taylor,
                      "H_exact": H_exact},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def _events_time(fn, steps, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def same_gpu_comparison(args, w, Rd, p, seed, bf16_value, stream):
    """The headline's comparison on the same GPU and matrix, measured in the
    same run: the plain FP64 estimator (Chebyshev + Taylor m, FP64 CUDA
    cores) and the learned low-degree form (BF16 degree-16 Chebyshev plus
    the correction network, trained here on sampled spectra), the latter
    against plain FP64 Chebyshev at degree 64, the degree it replaces.
    Accuracy reading for the learned form: its error from the exact entropy
    may exceed that of plain FP64 degree 64 by at most 1e-3 (relative)."""
    import torch

    import paper_1801_01072_gb300 as vne
    from paper_1801_01072_gb300 import learned

    m, s = w["m"], w["s"]
    H_exact = float(-(p[p > 0] * np.log(p[p > 0])).sum())
    f64 = lambda: vne.entropy_both(Rd, m, s, seed=seed, probe=w["probe"], precision="f64",
                                   power_iters=w["power_iters"])
    f64()
    f64_ms, f64_out = _events_time(f64, 2, stream)
    # learned form: train (outside every timed region), then time
    t0 = time.perf_counter()
    data = learned.spectral_samples(synth.learned_sample_params(args.learn_count, 1), s=s)
    theta0 = torch.tensor(synth.mlp_init(1), dtype=torch.float32).cuda()
    theta, _ = learned.train(theta0, data["features"], data["target"], epochs=args.learn_epochs,
                             batch=1024, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del data
    lf = lambda: learned.entropy_chebyshev_learned(Rd, theta, s=s, seed=seed, precision="bf16",
                                                   power_iters=w["power_iters"])
    for _ in range(3):
        lf()
    l_ms, l_out = _events_time(lf, 10, stream)
    c64 = lambda: vne.entropy_chebyshev(Rd, 64, s, seed=seed, probe="gaussian",
                                        precision="f64", power_iters=w["power_iters"],
                                        u_scale=1.05)
    c64_ms, c64_out = _events_time(c64, 1, stream)
    e_learned = abs(l_out.H - H_exact) / H_exact
    e_c64 = abs(c64_out.H - H_exact) / H_exact
    return {
        "fp64_same_workload": {"entropies_per_s": 1e3 / f64_ms, "ms": f64_ms,
                               "speedup_of_headline": bf16_value / (1e3 / f64_ms),
                               "H_chebyshev": f64_out.H_chebyshev, "H_taylor": f64_out.H_taylor},
        "learned_degree16_bf16": {
            "entropies_per_s": 1e3 / l_ms, "ms": l_ms, "rel_err_exact": e_learned,
            "H": l_out.H, "H_plain_degree16": l_out.H_plain,
            "training": {"spectra": args.learn_count, "epochs": args.learn_epochs,
                         "seconds_incl_sampling": train_s}},
        "fp64_chebyshev_degree64": {"entropies_per_s": 1e3 / c64_ms, "ms": c64_ms,
                                    "rel_err_exact": e_c64, "H": c64_out.H},
        "learned_speedup_over_fp64_degree64": c64_ms / l_ms,
        "learned_within_1e-3_of_fp64_degree64_accuracy": bool(e_learned <= e_c64 + 1e-3),
        "H_exact": H_exact,
    }


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1801_01072_gb300 as vne

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w, Rh, p = make_workload(args.workload)
    if w["kind"] == "lowrank":
        return run_gpu_projection(args, w, Rh, p, world, rank, local, dev)
    if w["kind"] == "learned":
        return run_gpu_learned(args, w, Rh, p, world, rank, local, dev)
    if w["kind"] == "batched":
        return run_gpu_batched(args, w, Rh, world, rank, local, dev)
    if w["kind"] == "hermitian":
        return run_gpu_hermitian(args, w, p, world, rank, local, dev)
    dense = w["kind"] == "dense"
    n, m, s = w["n"], w["m"], w["s"]
    prec = args.precision if dense else "f32"
    Rd = torch.as_tensor(Rh).to(dev)
    layout = "dense" if dense else "dia"
    seed = w["seed"] + 1000 * rank  # each rank: an independent estimate

    def step(R):
        if dense:
            return vne.entropy_both(R, m, s, seed=seed, probe=w["probe"], precision=prec,
                                    power_iters=w["power_iters"], layout=layout)
        return vne.entropy_chebyshev(R, m, s, seed=seed, probe=w["probe"], precision=prec,
                                     power_iters=w["power_iters"], layout=layout)

    h = vne._handle(local)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        out = step(Rd)
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    h.profile(True)
    n_launch0 = h.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            out = step(Rd)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    n_launch = h.launch_count() - n_launch0
    ms = ev0.elapsed_time(ev1)
    kind = 0 if (dense and prec.startswith("bf16")) else (1 if dense else 2)
    k_ms, k_n = h.profile_read(kind)
    p_ms, p_n = h.profile_read(3)  # power-method products
    h.profile(False)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())

    # ---- end to end: host-resident R, copies inside the call ----
    # (a) one single call per matrix: its copy, then its estimate
    Rpin = torch.as_tensor(Rh).pin_memory()
    step(Rpin)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    e2e_steps = max(3, args.steps // 4)
    for _ in range(e2e_steps):
        step(Rpin)
    ev3.record(stream)
    torch.cuda.synchronize()
    e2e_single_ms = max(ev2.elapsed_time(ev3) / e2e_steps,
                        (time.perf_counter() - e0) / e2e_steps * 1e3)
    # (b) the sequence call over host matrices (two pinned buffers,
    # alternating): each matrix's transfer runs while the previous one is
    # estimated; the first transfer is not hidden and is counted
    Rpin2 = Rpin.clone().pin_memory()
    seq_len = max(8, args.steps // 4)
    seq = [Rpin if i % 2 == 0 else Rpin2 for i in range(seq_len)]
    meth = "both" if dense else "chebyshev"

    def run_seq():
        return vne.entropy_sequence(seq, m, s, seed=seed, probe=w["probe"], precision=prec,
                                    power_iters=w["power_iters"], method=meth,
                                    layouts=[layout] * seq_len)
    seq_out = run_seq()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    ev2.record(stream)
    seq_out = run_seq()
    ev3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max(ev2.elapsed_time(ev3), (time.perf_counter() - e0) * 1e3) / seq_len
    # the sequence's estimates are the single call's
    one = step(Rpin)
    same = bool(np.all(seq_out[0] == (one.H_chebyshev if dense else one.H)))

    # ---- accuracy of this precision against the FP64 path on the GPU ----
    rel_err = None
    if rank == 0 and dense and prec != "f64" and not args.skip_f64_check:
        # the plain FP64 path on the same GPU, same probes: once with its own
        # power method (whole pipeline), once at this run's u (recurrence only)
        full = vne.entropy_both(Rd, m, s, seed=seed, probe=w["probe"], precision="f64",
                                power_iters=w["power_iters"])
        same_u = vne.entropy_both(Rd, m, s, seed=seed, probe=w["probe"], precision="f64",
                                  u=out.u)
        rel_err = {
            "chebyshev": abs(out.H_chebyshev - full.H_chebyshev) / abs(full.H_chebyshev),
            "taylor": abs(out.H_taylor - full.H_taylor) / abs(full.H_taylor),
            "chebyshev_same_u": abs(out.H_chebyshev - same_u.H_chebyshev) / abs(same_u.H_chebyshev),
            "taylor_same_u": abs(out.H_taylor - same_u.H_taylor) / abs(same_u.H_taylor),
            "u_rel_diff": abs(out.u - full.u) / full.u,
        }

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    step_ms = ms_max / args.steps
    value = world * args.steps / (ms_max / 1e3)
    pk, pk_src = peaks()
    if dense and prec in ("bf16", "bf16x3", "bf16x6", "f64", "f32"):
        # algorithmic flops per launch: 2 n^2 per probe column per step
        cols = 2 * s * m + s  # Chebyshev: m steps x s cols; Taylor: (m+1) steps x s cols
        flops = 2.0 * n * n * cols * args.steps
        achieved = flops / (k_ms / 1e3) / 1e12 if k_ms > 0 else None
        if prec.startswith("bf16"):
            # each launch is a few tens of microseconds inside a short timed
            # region: the burst peak applies
            peak = peak_value(pk, "bf16_tflops", "bf16_tflops_sustained")
            bound, unit = "tensor", "TFLOP/s"
        else:
            # CUDA-core peaks: FP32 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64 the
            # nominal 1.25 TFLOP/s (an FMA-chain probe measured 1.20)
            peak = 152 * 128 * 2 * 2.07e9 / 1e12 if prec == "f32" else 1.25
            bound, unit = "alu", "TFLOP/s"
        # DRAM bytes of one fused 256-column launch (ncu), when the source is unchanged
        traffic = profiled_traffic("k_tc_step_dense_n8192.md", "vne_tc.cu") \
            if (prec == "bf16" and args.workload == "dense_powerlaw_n8192") else None
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": (achieved / peak) if (achieved and peak) else None, "traffic": traffic,
                "kernel": "k_tc_step" if kind == 0 else "k_simt_step",
                "launches": k_n, "avg_launch_us": k_ms / max(k_n, 1) * 1e3,
                "peak_source": pk_src + " bf16 burst" if prec.startswith("bf16")
                else ("derived: FP32 lanes x 2 x max SM clock" if prec == "f32" else "nominal FP64")}
    else:
        # algorithmic bytes of the m banded steps of one estimate: every step reads
        # the band (4n(D)) and the packed signs (8n per 64 probes) and writes Y_t
        # (4ns); step t >= 2 reads Y_{t-1}; step t >= 3 also reads Y_{t-2}
        # (steps 1 and 2 take Y_0 from the signs)
        band_b = 4 * n * (w["half_bw"] + 1) + 8 * n * ((s + 63) // 64)
        y_b = 4 * n * s
        bytes_est = sum(band_b + y_b + (y_b if t >= 2 else 0) + (y_b if t >= 3 else 0)
                        for t in range(1, m + 1))
        achieved = bytes_est * args.steps / (k_ms / 1e3) / 1e9 if k_ms > 0 else None
        peak = peak_value(pk, "hbm_gbs")
        # DRAM bytes of one general step at n = 2e6 (ncu), scaled to this n
        # (the FP32 path with s = 64 runs the bulk-copy kernel of vne_dia_tma.cu)
        kname = "k_dia_step_tma" if prec == "f32" else "k_dia_step"
        tr = profiled_traffic("k_dia_step_tma_band_n2e6.md", "vne_dia_tma.cu") \
            if prec == "f32" else None
        traffic = int(tr * n / 2e6) if tr else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if (achieved and peak) else None, "traffic": traffic,
                "kernel": kname, "launches": k_n,
                "avg_launch_us": k_ms / max(k_n, 1) * 1e3, "peak_source": pk_src + " hbm"}

    cpu = None
    if world == 1 and not args.skip_cpu:
        if dense:
            t_full, desc, threads = oracle_full_time(w, Rh)
        else:
            t_full, desc, threads = oracle_sample_time(w, Rh, min(args.cpu_probes, 2))
        cpu = {"value": 1.0 / t_full, "unit": "entropies/s", "cores": threads, "kind": "oracle",
               "sample": desc}

    # the plain FP64 estimator and the learned low-degree form on the same GPU
    extras = None
    if dense and prec == "bf16" and not args.skip_extras and args.workload == "dense_powerlaw_n8192":
        extras = same_gpu_comparison(args, w, Rd, p, seed, value, stream)

    clocks = clk.summary()
    line = {
        "metric": "entropies/s (density matrices through power method + Chebyshev m=40 + "
                  "Taylor m=40, s=128) at <=1e-3 rel. error vs the FP64 path on the same GPU"
                  if dense else "entropies/s (banded Chebyshev m=30, s=64)",
        "value": value,
        "unit": "entropies/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"bf16": "bf16", "bf16x3": "bf16x3", "bf16x6": "bf16x6", "f64": "f64",
                  "f32": "f32"}[prec],
        "data": "synthetic (seeded density matrices, no dataset)",
        "config": {"workload": args.workload, "n": n, "m": m, "s": s, "probe": w["probe"],
                   "power_iters": w["power_iters"], "precision": prec,
                   "estimators": "chebyshev+taylor" if dense else "chebyshev",
                   "input": "R FP64 resident in HBM" if dense else "band FP32 resident in HBM",
                   "l2": "inputs larger than L2 (R is %.0f MB)" % (Rh.nbytes / 1e6),
                   "parallelism": f"independent matrices, {world} GPU(s)"},
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "entropies/s",
                "h2d_bytes_per_step": int(Rh.nbytes), "d2h_bytes_per_step": 200 * 8,
                "api": f"entropy_sequence over {seq_len} pinned host matrices (two buffers, "
                       "alternating): each transfer overlaps the previous estimate",
                "equals_single_calls": same,
                "single_call": {"value": world * 1e3 / e2e_single_ms, "unit": "entropies/s",
                                "api": "entropy_both / entropy_chebyshev on one pinned host "
                                       "matrix: copy, then estimate"}},
        "gpu_launches": int(n_launch),
        "phases_ms_per_step": {"recurrence": k_ms / args.steps, "power_method": p_ms / args.steps,
                               "other": ms_max / args.steps - (k_ms + p_ms) / args.steps},
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "rel_err_vs_f64": rel_err,
        "vs_plain_fp64_same_gpu": extras,
        "estimates": {"H_chebyshev": getattr(out, "H_chebyshev", getattr(out, "H", None)),
                      "H_taylor": getattr(out, "H_taylor", None), "u": out.u,
                      "H_exact": float(-(p[p > 0] * np.log(p[p > 0])).sum()) if p is not None
                      else None},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------

def run_reference_projection(args, w, Rh):
    times = []
    for i in range(args.warmup + args.steps):
        t, desc, threads = oracle_projection_time(w, Rh)
        if i >= args.warmup:
            times.append(t)
    value = len(times) / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": PROJ_METRIC if not w.get("krylov", 0) else KRYLOV_METRIC,
        "value": value, "unit": "entropies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded rank-k density matrices, no dataset)",
        "config": {"workload": args.workload, "n": w["n"], "k": w["k"], "s": w["s"],
                   "sketch": w["sketch"]},
        "cpu_baseline": {"value": value, "unit": "entropies/s", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "entropies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def run_reference_batched(args, w, specs):
    import oracle as O
    from oracle import rng

    idx = list(range(0, len(specs), max(1, len(specs) // 4)))[:4]
    mats = [synth.dense_density(synth.haar_orthogonal(specs[i][0], specs[i][2]), specs[i][1])
            for i in idx]
    times = []
    for it in range(args.warmup + args.steps):
        tot = 0.0
        for R, i in zip(mats, idx):
            n = specs[i][0]
            t0 = time.perf_counter()
            lam, _ = O.power_method(R, rng.power_start(n, 1, w["seed"]), w["power_iters"])
            t1 = time.perf_counter()
            G = rng.probes(n, w["s"], w["seed"], w["probe"])[:, :4]
            O.chebyshev_moments(R, G, O.interval_u(lam, 1.0), w["m"])
            tot += (t1 - t0) + (time.perf_counter() - t1) * w["s"] / 4
        if it >= args.warmup:
            times.append(tot / len(idx))
    value = len(times) / sum(times)
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count() or 1
    desc = (f"oracle (NumPy FP64) on {len(idx)} of the {len(specs)} matrices: power method + "
            f"Chebyshev m={w['m']} on 4 of the s={w['s']} probes, recurrence scaled by s/4, "
            f"mean time per matrix")
    print(json.dumps({
        "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": "entropies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded uneven density matrices, no dataset)",
        "config": {"workload": args.workload, "count": len(specs), "m": w["m"], "s": w["s"]},
        "cpu_baseline": {"value": value, "unit": "entropies/s", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "entropies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def run_reference_hermitian(args, w, p):
    import oracle.hermitian as OH
    from oracle import rng

    n, m, s = w["n"], w["m"], w["s"]
    R = synth.hermitian_density(n, p, w["seed"])
    sp = 2
    G = rng.gaussian(n, s, w["seed"])[:, :sp]
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        OH.chebyshev_moments_complex(R, G, 1.0, m)
        OH.taylor_terms_complex(R, G, 1.0, m)
        if it >= args.warmup:
            times.append((time.perf_counter() - t0) * s / sp)
    value = len(times) / sum(times)
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count() or 1
    desc = (f"oracle (NumPy complex128) Chebyshev + Taylor recurrences m={m} on {sp} of the "
            f"s={s} probes of the full n={n} matrix, scaled by s/{sp}")
    print(json.dumps({
        "impl": "reference", "metric": HERM_METRIC, "value": value, "unit": "entropies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded complex density matrix, no dataset)",
        "config": {"workload": args.workload, "n": n, "m": m, "s": s, "u": 1.0},
        "cpu_baseline": {"value": value, "unit": "entropies/s", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "entropies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, Rh, p = make_workload(args.workload)
    if w["kind"] == "batched":
        return run_reference_batched(args, w, Rh)
    if w["kind"] == "hermitian":
        return run_reference_hermitian(args, w, p)
    if w["kind"] == "lowrank":
        return run_reference_projection(args, w, Rh)
    if w["kind"] == "learned":
        w = dict(w, kind="dense_cheb")
    times = []
    for i in range(args.warmup + args.steps):
        if w["kind"] in ("dense", "dense_cheb"):
            # a whole oracle estimate per step (all probes, nothing scaled)
            t, desc, threads = oracle_full_time(w, Rh)
        else:
            t, desc, threads = oracle_sample_time(w, Rh, args.ref_probes)
        if i >= args.warmup:
            times.append(t)
    tot = sum(times)
    value = len(times) / tot
    line = {
        "impl": "reference",
        "metric": LEARNED_METRIC if w["kind"] == "dense_cheb" else
                  "entropies/s (density matrices through power method + Chebyshev m=40 + "
                  "Taylor m=40, s=128) at <=1e-3 rel. error vs the FP64 path on the same GPU"
                  if w["kind"] == "dense" else "entropies/s (banded Chebyshev m=30, s=64)",
        "value": value,
        "unit": "entropies/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot / len(times) * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded density matrices, no dataset)",
        "config": {"workload": args.workload, "n": w["n"], "m": w["m"], "s": w["s"],
                   "probe": w["probe"], "power_iters": w["power_iters"]},
        "cpu_baseline": {"value": value, "unit": "entropies/s", "cores": threads,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "entropies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dense_powerlaw_n8192", choices=list(synth.WORKLOADS))
    ap.add_argument("--precision", default="bf16", choices=["bf16", "bf16x3", "bf16x6", "f64", "f32"],
                    help="recurrence arithmetic; the projection workloads run bf16x3 unless f32, "
                         "f64 or bf16x6 is given")
    ap.add_argument("--cpu-probes", type=int, default=16)
    ap.add_argument("--ref-probes", type=int, default=4)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-f64-check", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the same-GPU FP64 and learned-form comparison of the headline")
    ap.add_argument("--learn-count", type=int, default=100000,
                    help="training spectra of the learned form in the headline comparison")
    ap.add_argument("--learn-epochs", type=int, default=20)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
