#!/usr/bin/env python
"""Benchmark of the lattice Green's function step on one GB300.

Workload: the Ce-like f-system (N_k = 1000 k-points, band window N_b = 40,
m = 14 correlated orbitals, 1024 positive Matsubara frequencies at beta = 100,
U = 6 eV), seeded synthetic inputs, FP64 path.

One step is one pass of the whole hot path over the workload, as a DMFT
iteration needs it:
  1. mu search: Newton from mu = 0 on N(mu) (each evaluation embeds and inverts
     every G(k, i w_n) and sums the Matsubara series),
  2. one fused pass at mu*: G_loc, rho_k, N, dN/dmu, n_corr,
  3. the adjoint at mu*: Sigma_bar and mu_bar for a seeded G_loc_bar and N_bar = 1.
value = (k, i w_n) points evaluated per second (every pass counts its points).

The same line carries, beside the FP64 headline: the mixed-precision step
(FP32 inverse, FP64 sums, refined projections) and the FP32-pair step on the
same workload; the low-rank (eigenbasis) algorithm; the NiO-like workload
(N_k = 4096, N_b = 96, m = 20, 2048 frequencies): one fixed-mu fused pass on
the FP64 and on the mixed path and the mixed mu search, with errors against
the oracle; and the batched workload (8 systems, ragged windows of 48-128
bands, complex128 and complex64 inputs in one context) on both paths.

``--impl reference`` times the FP64 CPU oracle (the plain definition, one LU
inverse per point) on the host cores instead, on a bounded sample of the same
workload, and prints the same JSON line with "impl": "reference".
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "(k,iω_n) G points/s & % FP64/TF32 peak; mixed vs plain FP64 GPU at 1e-7 N(μ)"
UNIT = "points/s"
WORKLOAD = "ce_like: N_k=1000, N_b=40, m=14, N_w=1024, beta=100 1/eV, U=6 eV, dense H, two-pole Sigma"
# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Peak of the FP32-pair arithmetic (GF_PREC_PAIR), in FP64-equivalent flop/s: the FP32 pipes
# issue 152 SMs x 128 lanes x 2.07 GHz operations, and one FP32-pair complex multiply-add takes
# at least 48 of them (4 error-free products with head sums, 12 operations each); 8 flop per CMAC.
MIXED_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 48 * 8 / 1e12
L2_FLUSH_BYTES = 256 << 20
PROFILES = ROOT / "profiles"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--no-nio", action="store_true", help="skip the NiO-like leg of the default line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched leg of the default line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the bounded CPU-oracle sample")
    ap.add_argument("--nk-scale", type=float, default=1.0,
                    help="batched workload: fraction of each system's k-points")
    ap.add_argument("--nk", type=int, default=None,
                    help="smaller k-set of the same workload (profiling captures only)")
    ap.add_argument("--n-iw", type=int, default=None,
                    help="fewer Matsubara frequencies (profiling captures only)")
    ap.add_argument("--precision", choices=["fp64", "mixed", "pair"], default="fp64",
                    help="arithmetic of the point kernel (mixed: FP32 inverse with refined "
                         "projections; pair: FP32 pairs on the FP32 pipes)")
    ap.add_argument("--workload", choices=["ce_like", "nio_like", "batched", "adjoint", "lowrank",
                                           "pole", "dmft_step", "passes"],
                    default="ce_like", help="non-default workloads print one measurement line each")
    ap.add_argument("--system", choices=["nio_like", "ce_like"], default="nio_like",
                    help="--workload passes: the shapes to run (with --nk / --n-iw)")
    ap.add_argument("--peaks", action="store_true",
                    help="compile and run the pipe-throughput microbenchmark (peaks.cu) and exit")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.TemporaryFile(mode="w+")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


def ncu_traffic():
    """dram bytes per launch of the point kernel from the committed ncu summary (or None)."""
    f = PROFILES / "point_fp64_ce_like.md"
    if not f.exists():
        return None
    for line in f.read_text().splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_calibrate(system, mu):
    """Seconds per k-point of the FP64 oracle's Matsubara-sum pass (all frequencies)."""
    import oracle
    o = oracle.get()
    o.set_threads(cpu_cores())
    s = system
    kc = min(s.nk, o.get_threads())
    w = np.full(s.nk, 1.0 / s.nk)
    t0 = time.perf_counter()
    o.density(s.H[:kc], s.P[:kc], s.sigma, s.sigma_inf, s.beta, mu, weights=w[:kc], want_rho=False)
    return max(time.perf_counter() - t0, 1e-6) / kc


def oracle_sample(system, mu, seconds):
    """Time the FP64 oracle's Matsubara-sum pass on the first K k-points (K sized to ~seconds)."""
    import oracle
    o = oracle.get()
    s = system
    per_k = oracle_calibrate(s, mu)
    thr = o.get_threads()
    k = int(min(s.nk, max(thr, int(seconds / per_k) // thr * thr)))
    w = np.full(s.nk, 1.0 / s.nk)
    t0 = time.perf_counter()
    o.density(s.H[:k], s.P[:k], s.sigma, s.sigma_inf, s.beta, mu, weights=w[:k], want_rho=False)
    dt = time.perf_counter() - t0
    pts = k * s.n_iw
    return {"value": pts / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{k} of {s.nk} k-points x all {s.n_iw} frequencies, one Matsubara-sum "
                      f"pass (LU inverse per point, N and dN/dmu) at fixed mu, {dt:.1f} s"}, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1111_2157_gb300 import synth
    s = synth.ce_like().systems[0]
    import oracle
    o = oracle.get()
    o.set_threads(cpu_cores())
    per_step = max(2.0, min(10.0, 100.0 / max(1, args.steps + args.warmup)))
    per_k = oracle_calibrate(s, 0.0)
    thr = o.get_threads()
    k = int(min(s.nk, max(thr, int(per_step / per_k) // thr * thr)))
    w = np.full(s.nk, 1.0 / s.nk)
    for _ in range(args.warmup):
        o.density(s.H[:k], s.P[:k], s.sigma, s.sigma_inf, s.beta, 0.0, weights=w[:k], want_rho=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.density(s.H[:k], s.P[:k], s.sigma, s.sigma_inf, s.beta, 0.0, weights=w[:k], want_rho=False)
    dt = time.perf_counter() - t0
    value = args.steps * k * s.n_iw / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32", "pair": "f32x2"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"oracle Matsubara-sum pass over {k} k-points x "
                                                     f"{s.n_iw} frequencies at mu=0 (bounded sample)",
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.get_threads(), "kind": "oracle",
                             "sample": f"{k} of {s.nk} k-points x all {s.n_iw} frequencies per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_peaks():
    """Build peaks.cu (beside this script) with nvcc and run it (prints one line per pipe)."""
    from paper_1111_2157_gb300 import build as gfbuild
    src = ROOT / "peaks.cu"
    exe = gfbuild.BUILD / "peaks"
    gfbuild.BUILD.mkdir(exist_ok=True)
    subprocess.run([gfbuild.nvcc(), *gfbuild.ARCH, "-O3", "-o", str(exe), str(src)], check=True)
    return subprocess.run([str(exe)]).returncode


def _sync_time(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def _pack(blocks):
    return np.concatenate([np.asarray(b).reshape(-1) for b in blocks])


def _context(gf, systems, precision, graph=False, lowrank=False):
    g = gf.GreensFunction.for_systems(systems, precision=precision, graph=graph, lowrank=lowrank)
    g.set_hamiltonian(_pack([_pack(s.H) for s in systems]))
    g.set_projectors(_pack([_pack(s.P) for s in systems]))
    g.set_sigma(_pack([s.sigma for s in systems]), _pack([s.sigma_inf for s in systems]))
    return g


def _lr_pole_cases(args, synth):
    """Ce-like and a NiO-like k-subset; with --nk / --n-iw only a small Ce-like case (profiling)."""
    if args.nk or args.n_iw:
        return [("ce_like_small", synth.ce_like(nk=args.nk or 1000, n_iw=args.n_iw or 1024).systems[0])]
    return [("ce_like", synth.ce_like().systems[0]),
            ("nio_like_1024k", synth.nio_like(nk=1024).systems[0])]


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
MIXED_MU_TOL = 1e-8  # mixed path: mu search to |N - N_target| <= 1e-8 N_target (FP32 noise ~1e-9)


def _dev_context(gf, systems, precision, graph=False, lowrank=False, input_dtype="c128"):
    """Context with the inputs uploaded from device tensors (resident in HBM); with
    input_dtype="per_system" each system is uploaded in its own dtype (complex64 systems
    as complex64)."""
    import torch
    g = gf.GreensFunction.for_systems(systems, precision=precision, graph=graph, lowrank=lowrank,
                                      input_dtype=input_dtype)
    g.set_hamiltonian(torch.from_numpy(_pack([_pack(s.H) for s in systems])).cuda())
    g.set_projectors(torch.from_numpy(_pack([_pack(s.P) for s in systems])).cuda())
    g.set_sigma(torch.from_numpy(_pack([s.sigma for s in systems])).cuda(),
                torch.from_numpy(_pack([s.sigma_inf for s in systems])).cuda())
    return g


def nio_leg(gf, synth, o, nk=4096, n_iw=2048):
    """NiO-like precision workload: one fixed-mu fused pass (G_loc, N, dN/dmu) on the FP64
    and on the mixed path, the mixed mu search, and errors against the oracle."""
    s = synth.nio_like(nk=nk, n_iw=n_iw).systems[0]
    npts = s.nk * s.n_iw
    out = {"config": f"N_k={s.nk}, N_b=96, m=20 (2 atoms x 5 d x 2 spin, AFM Sigma), N_w={s.n_iw}, "
                     "beta=40 1/eV, U=8 eV", "points_per_pass": npts}
    # mixed: mu search (graph replay of the N(mu) evaluation), then the fused pass at mu*
    gm = _dev_context(gf, [s], "mixed", graph=True)
    tol = MIXED_MU_TOL * s.n_target
    (mu, it), t_mu = _sync_time(lambda: gm.find_mu([s.n_target], 0.0, tol=tol))
    smu = gm.stats()
    gm.evaluate(mu, rho=False, n_corr=False)  # autotunes the fused pass's launch
    evm, t_m = _sync_time(lambda: gm.evaluate(mu, rho=False, n_corr=False))
    stm = gm.stats()
    gl_m = evm["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    mixed_log = gm.tuning_log()
    gm.close()
    # FP64: the same fused pass (one call; the autotuner's samples are outside its kernel time)
    g64 = _dev_context(gf, [s], "fp64")
    ev64, t_64 = _sync_time(lambda: g64.evaluate(mu, rho=False, n_corr=False))
    st64 = g64.stats()
    gl_d = ev64["gloc"].cpu().numpy().reshape(s.n_iw, s.m, s.m)
    fp64_log = g64.tuning_log()
    g64.close()
    idx = [0, 1, s.n_iw // 2, s.n_iw - 1]
    glo = o.local(s.H, s.P, s.sigma, s.beta, float(mu[0]), n_idx=idx)
    # N against the oracle on an 8-k subset (all frequencies), the GPU evaluating the same subset
    ks = list(range(8))
    sub = synth.System(s.H[ks], s.P[ks], s.pole, s.sigma, s.beta, s.n_target)
    r_o = o.density(sub.H, sub.P, sub.sigma, sub.sigma_inf, sub.beta, float(mu[0]), want_rho=False)
    gs = _dev_context(gf, [sub], "mixed")
    n_sub, dn_sub = gs.occupation(mu)
    gs.close()
    k_m, k_d = stm["kernel_ms"] / 1e3, st64["kernel_ms"] / 1e3
    # the N(mu) pass at mu* on the tcgen05 tensor-core kernel (selected with GF_KERNEL=tc)
    # beside the FP32 register kernel; N against the FP64 pass
    n64 = float(ev64["N"][0])
    tcl = {}
    for kern in ("tc", "f32r"):
        os.environ["GF_KERNEL"] = kern
        try:
            gk = _dev_context(gf, [s], "mixed")
            gk.occupation(mu)  # the first call autotunes
            (n_k, _), t_k = _sync_time(lambda: gk.occupation(mu))
            stk = gk.stats()
            tcl[kern] = {"pass_s": t_k, "pass_kernel_s": stk["kernel_ms"] / 1e3,
                         "points_per_s": npts / (stk["kernel_ms"] / 1e3),
                         "alg_tflops": stk["flops"] / stk["kernel_ms"] / 1e9,
                         "N_rel_err_vs_fp64_gpu": abs(float(n_k[0]) - n64) / n64,
                         "kernel_choice": gk.tuning_log()}
            gk.close()
        finally:
            del os.environ["GF_KERNEL"]
    tcl["tc_speed_vs_f32r"] = tcl["f32r"]["pass_kernel_s"] / tcl["tc"]["pass_kernel_s"]
    out.update({
        "mu_star": float(mu[0]), "N_at_mu_star": float(evm["N"][0]),
        "N_pass_tensor_core_vs_fp32_kernel": tcl,
        "fp64": {"pass_s": t_64, "pass_kernel_s": k_d, "points_per_s": npts / k_d,
                 "kernel_tflops": st64["flops"] / st64["kernel_ms"] / 1e9,
                 "frac_of_fp64_peak": st64["flops"] / st64["kernel_ms"] / 1e9 / FP64_PEAK_TFLOPS,
                 "kernel_choice": fp64_log},
        "mixed": {"pass_s": t_m, "pass_kernel_s": k_m, "points_per_s": npts / k_m,
                  "speedup_vs_fp64_gpu": k_d / k_m, "speedup_vs_fp64_gpu_wall": t_64 / t_m,
                  "roofline": {"bound": "alu", "achieved": stm["flops"] / stm["kernel_ms"] / 1e9,
                               "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": stm["flops"] / stm["kernel_ms"] / 1e9 / FP32_PEAK_TFLOPS,
                               "kernel": "k_point_f32r (autotuned tiles)",
                               "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"},
                  "find_mu_s": t_mu, "find_mu_evaluations": it,
                  "find_mu_points_per_s": smu["points"] / t_mu,
                  "find_mu_speedup_vs_fp64_pass_rate": (smu["points"] / t_mu) / (npts / k_d),
                  "kernel_choice": mixed_log},
        "N_rel_err_mixed_vs_fp64_gpu": abs(float(evm["N"][0]) - float(ev64["N"][0])) / float(ev64["N"][0]),
        "dN_dmu_rel_err_mixed_vs_fp64_gpu": abs(float(evm["dN_dmu"][0]) - float(ev64["dN_dmu"][0]))
                                             / float(ev64["dN_dmu"][0]),
        "G_loc_rel_err_mixed_vs_fp64_gpu": float(np.max(np.abs(gl_m - gl_d)) / np.max(np.abs(gl_d))),
        "G_loc_rel_err_vs_oracle": {"mixed": float(np.max(np.abs(gl_m[idx] - glo)) / np.max(np.abs(glo))),
                                    "fp64": float(np.max(np.abs(gl_d[idx] - glo)) / np.max(np.abs(glo))),
                                    "sample": f"frequencies {idx} over all {s.nk} k-points"},
        "N_rel_err_vs_oracle": {"mixed": abs(float(n_sub[0]) - r_o["N"]) / r_o["N"],
                                "sample": "k-points 0-7, all frequencies, at mu*"},
    })
    return out


def _as_uploaded(synth, s):
    """A complex64 system as the library receives it (inputs rounded to complex64)."""
    if s.dtype != "c64":
        return s
    r = lambda a: np.asarray(a).astype(np.complex64).astype(np.complex128)  # noqa: E731
    H = [r(h) for h in s.H] if isinstance(s.H, list) else r(s.H)
    P = [r(p) for p in s.P] if isinstance(s.P, list) else r(s.P)
    return synth.System(H, P, synth.PoleSigma(r(s.pole.sigma_inf), s.pole.p, s.pole.V), r(s.sigma),
                        s.beta, s.n_target, dtype="c64")


def batched_leg(gf, synth, o, nk_scale=1.0):
    """Batched workload: 8 systems with ragged windows, half of them complex64 and half
    complex128, in one context and one launch per window bucket: FP64 and mixed N(mu) passes,
    one launch per system, and a graph-replayed mixed mu search."""
    systems = synth.batched(nk_scale=nk_scale).systems
    pd = "per_system"
    pts = sum(sy.nk * sy.n_iw for sy in systems)
    mus = [0.0] * len(systems)
    out = {"config": (f"8 systems, N_k per system {[sy.nk for sy in systems]}, N_b(k) uniform in [48, 128], "
                      f"m {[sy.m for sy in systems]}, N_w=1024, beta=40 (k-sets x {nk_scale}); inputs "
                      f"{[sy.dtype for sy in systems]} in one context"),
           "points_per_pass": pts}
    g64 = _dev_context(gf, systems, "fp64", input_dtype=pd)
    (n64, d64), t64 = _sync_time(lambda: g64.occupation(mus))
    s64 = g64.stats()
    out["fp64"] = {"pass_s": t64, "pass_kernel_s": s64["kernel_ms"] / 1e3,
                   "points_per_s": pts / (s64["kernel_ms"] / 1e3), "launches": s64["launches"],
                   "kernel_tflops": s64["flops"] / s64["kernel_ms"] / 1e9}
    g64.close()
    gm = _dev_context(gf, systems, "mixed", input_dtype=pd)
    gm.occupation(mus)
    (nm, dm), tm = _sync_time(lambda: gm.occupation(mus))
    sm_ = gm.stats()
    log = gm.tuning_log()
    gm.close()
    t_per, n_launch = 0.0, 0
    for sy in systems:
        gi = _dev_context(gf, [sy], "mixed", input_dtype=pd)
        gi.occupation([0.0])
        _, t = _sync_time(lambda: gi.occupation([0.0]))
        t_per += t
        n_launch += gi.stats()["launches"]
        gi.close()
    gg = _dev_context(gf, systems, "mixed", graph=True, input_dtype=pd)
    targets = [sy.n_target for sy in systems]
    (mu_g, it_g), t_g = _sync_time(lambda: gg.find_mu(targets, 0.0, tol=MIXED_MU_TOL * min(targets)))
    pts_g = gg.stats()["points"]
    gg.close()
    # N against the oracle on k-subsets of two systems (4 k-points each, all frequencies)
    errs = []
    for i in (0, 1):
        sy = systems[i]
        sub = synth.System(sy.H[:4], sy.P[:4], sy.pole, sy.sigma, sy.beta, sy.n_target, dtype=sy.dtype)
        up = _as_uploaded(synth, sub)
        r_o = o.density(up.H, up.P, up.sigma, up.sigma_inf, up.beta, 0.0, want_rho=False)
        gs = _dev_context(gf, [sub], "mixed", input_dtype=pd)
        n_s, _ = gs.occupation([0.0])
        gs.close()
        errs.append(abs(float(n_s[0]) - r_o["N"]) / r_o["N"])
    k_m = sm_["kernel_ms"] / 1e3
    out["mixed"] = {"pass_s": tm, "pass_kernel_s": k_m, "points_per_s": pts / k_m,
                    "launches": sm_["launches"], "speedup_vs_fp64_gpu": s64["kernel_ms"] / sm_["kernel_ms"],
                    "roofline": {"bound": "alu", "achieved": sm_["flops"] / sm_["kernel_ms"] / 1e9,
                                 "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": sm_["flops"] / sm_["kernel_ms"] / 1e9 / FP32_PEAK_TFLOPS},
                    "per_system_launches_s": t_per, "per_system_kernel_launches": n_launch,
                    "speedup_one_launch_vs_per_system": t_per / tm,
                    "graph_find_mu_s": t_g, "graph_find_mu_evaluations": it_g,
                    "graph_find_mu_points_per_s": pts_g / t_g, "kernel_choice": log}
    out["N_rel_err_mixed_vs_fp64_gpu"] = float(np.max(np.abs(nm - n64) / n64))
    out["dN_dmu_rel_err_mixed_vs_fp64_gpu"] = float(np.max(np.abs(dm - d64) / d64))
    out["N_rel_err_vs_oracle"] = {"mixed": max(errs), "sample": "systems 0 (complex128) and 1 (complex64), "
                                                                 "k-points 0-3 each, all frequencies, mu = 0"}
    return out


def run_workload(args):
    """Measurements on the NiO-like, batched and adjoint workloads (one JSON line each)."""
    import torch
    from paper_1111_2157_gb300 import build as gfbuild
    if not gfbuild.LIB.exists():
        gfbuild.build()
    from paper_1111_2157_gb300 import gf, synth
    import oracle
    o = oracle.get()
    o.set_threads(cpu_cores())
    out = {"workload": args.workload}
    if args.workload == "nio_like":
        out.update(nio_leg(gf, synth, o, nk=args.nk or 4096, n_iw=args.n_iw or 2048))
    elif args.workload == "passes":
        # one N(mu) pass and one fused G_loc + N pass of the point kernel of --precision
        # (profiling captures; GF_KERNEL=tc puts the mixed N(mu) pass on the tensor cores)
        kw = {k: v for k, v in (("nk", args.nk), ("n_iw", args.n_iw)) if v}
        s = (synth.nio_like(**kw) if args.system == "nio_like" else synth.ce_like(**kw)).systems[0]
        g = _dev_context(gf, [s], args.precision)
        res = {}
        for name, call in (("occupation", lambda: g.occupation([0.1])),
                           ("fused_gloc_N", lambda: g.evaluate([0.1], rho=False, n_corr=False))):
            _, t = _sync_time(call)
            st = g.stats()
            res[name] = {"s": t, "kernel_s": st["kernel_ms"] / 1e3,
                         "points_per_s": st["points"] / (st["kernel_ms"] / 1e3),
                         "alg_tflops": st["flops"] / st["kernel_ms"] / 1e9}
        out.update({"config": f"{args.system}: N_k={s.nk}, N_b={s.H.shape[-1]}, m={s.m}, N_w={s.n_iw}",
                    "passes": res, "kernel_choice": g.tuning_log()})
        g.close()
    elif args.workload == "batched":
        out.update(batched_leg(gf, synth, o, nk_scale=args.nk_scale))
    elif args.workload == "adjoint":
        from paper_1111_2157_gb300.autograd import lattice_green, newton_mu
        s = synth.adjoint_case().systems[0]
        out["config"] = "N_k=2048, N_b=64, m=14, N_w=1024, beta=100 (Ce-like generators)"
        rng = np.random.default_rng(5)
        gbar = torch.from_numpy(rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)).cuda()
        for prec in ("fp64", "mixed"):
            g = _context(gf, [s], prec)
            sigma = torch.tensor(s.sigma, dtype=torch.complex128, device="cuda", requires_grad=True)
            mu = torch.tensor([0.2], dtype=torch.float64, requires_grad=True)
            (gl, n), t_f = _sync_time(lambda: lattice_green(g, sigma, mu, s.sigma_inf))
            loss = (torch.conj(gbar) * gl).real.sum() + 0.7 * n.sum()
            _, t_b = _sync_time(lambda: loss.backward())
            ntol = MIXED_MU_TOL * s.n_target if prec == "mixed" else 1e-10  # above the FP32 noise of N
            (mu_n, it), t_n = _sync_time(lambda: newton_mu(g, sigma.detach(), s.sigma_inf, s.n_target, 0.0,
                                                           tol=ntol))
            out[prec] = {"forward_s": t_f, "backward_s": t_b, "newton_mu": mu_n, "newton_evaluations": it,
                         "newton_tol": ntol,
                         "newton_s": t_n, "grad_sample": [complex(sigma.grad[0, 0, 0].item()).real,
                                                          float(mu.grad.item())]}
            if prec == "fp64":
                h = 1e-6
                sig0 = sigma.detach()
                fd = []
                for (w, a, b) in [(0, 0, 0), (511, 3, 9)]:
                    val = 0j
                    for unit in (1.0, 1j):
                        sp, sm = sig0.clone(), sig0.clone()
                        sp[w, a, b] += h * unit
                        sm[w, a, b] -= h * unit
                        lp = lattice_green(g, sp, mu.detach(), s.sigma_inf)
                        lm = lattice_green(g, sm, mu.detach(), s.sigma_inf)
                        fp_ = float(((torch.conj(gbar) * lp[0]).real.sum() + 0.7 * lp[1].sum()).item())
                        fm_ = float(((torch.conj(gbar) * lm[0]).real.sum() + 0.7 * lm[1].sum()).item())
                        val += unit * (fp_ - fm_) / (2 * h)
                    got = complex(sigma.grad[w, a, b].item())
                    fd.append({"entry": [w, a, b], "adjoint": [got.real, got.imag], "fd": [val.real, val.imag],
                               "rel_err": abs(got - val) / abs(val)})
                out["fp64"]["finite_differences"] = fd
                grad64 = sigma.grad.detach().clone()
                mug64 = float(mu.grad.item())
            else:
                out["mixed"]["grad_rel_err_vs_fp64_gpu"] = float((sigma.grad - grad64).abs().max() / grad64.abs().max())
                out["mixed"]["mu_grad_rel_err_vs_fp64_gpu"] = abs(mu.grad.item() - mug64) / abs(mug64)
            g.close()
        # oracle gradient on a k-subset (same weights as the full problem's first 16 k-points)
        ks = list(range(16))
        w = np.full(16, 1.0 / 16)
        sb_o, mb_o = o.backward(s.H[ks], s.P[ks], s.sigma, s.sigma_inf, s.beta, 0.2,
                                gloc_bar=gbar.cpu().numpy(), n_bar=0.7, weights=w)
        sub = synth.System(s.H[ks], s.P[ks], s.pole, s.sigma, s.beta, s.n_target)
        gsub = _context(gf, [sub], "fp64")
        sb_g, mb_g = gsub.backward([0.2], gloc_bar=gbar.reshape(-1), n_bar=[0.7])
        out["oracle_gradient_16k"] = {"sigma_bar_rel_err": float(np.max(np.abs(sb_g.cpu().numpy() - sb_o.reshape(-1)))
                                                                 / np.max(np.abs(sb_o))),
                                      "mu_bar_rel_err": abs(mb_g[0] - mb_o) / abs(mb_o)}
        gsub.close()
    elif args.workload == "lowrank":
        # eigenbasis (Woodbury) algorithm against the direct inverse, FP64, at fixed mu
        out["config"] = ("Ce-like full size; NiO-like with N_k = 1024 of its 4096 k-points; the batched "
                         f"workload with its k-sets scaled by {args.nk_scale}")
        cases = [(name, [s]) for name, s in _lr_pole_cases(args, synth)]
        if not (args.nk or args.n_iw):
            cases.append(("batched", synth.batched(nk_scale=args.nk_scale).systems))
        for name, systems in cases:
            mu = [0.3] * len(systems)
            gd = _context(gf, systems, "fp64")
            gl = _context(gf, systems, "fp64", lowrank=True)
            gd.occupation(mu)
            (nd, dd), td = _sync_time(lambda: gd.occupation(mu))
            sd = gd.stats()
            _, t_setup = _sync_time(lambda: gl.occupation(mu))  # includes the eigen-decomposition
            (nl, dl), tl = _sync_time(lambda: gl.occupation(mu))
            sl = gl.stats()
            pts = sum(s.nk * s.n_iw for s in systems)
            # the same with GF_PREC_MIXED: FP32-pair band sums, FP64 m x m algebra
            gx = _context(gf, systems, "mixed", lowrank=True)
            gx.occupation(mu)
            (nx, dx), tx = _sync_time(lambda: gx.occupation(mu))
            gx.close()
            res = {
                "points": pts,
                "mixed_lowrank_occupation_s": tx,
                "mixed_lowrank_speedup_vs_lowrank": tl / tx,
                "mixed_lowrank_speedup_vs_direct_fp64": td / tx,
                "mixed_lowrank_N_rel_diff_vs_direct": float(np.max(np.abs(nx - nd) / nd)),
                "mixed_lowrank_dN_rel_diff_vs_direct": float(np.max(np.abs(dx - dd) / dd)),
                "direct_occupation_s": td, "lowrank_occupation_s": tl,
                "lowrank_first_call_s_with_eigendecomposition": t_setup,
                "speedup_occupation": td / tl,
                "lowrank_points_per_s": pts / tl, "direct_points_per_s": pts / td,
                "lowrank_kernel_tflops": sl["flops"] / sl["kernel_ms"] / 1e9,
                "lowrank_frac_of_fp64_peak": sl["flops"] / sl["kernel_ms"] / 1e9 / FP64_PEAK_TFLOPS,
                "direct_kernel_tflops": sd["flops"] / sd["kernel_ms"] / 1e9,
                "N_rel_diff": float(np.max(np.abs(nl - nd) / nd)),
                "dN_rel_diff": float(np.max(np.abs(dl - dd) / dd))}
            if len(systems) == 1:
                s = systems[0]
                ed, t_ed = _sync_time(lambda: gd.evaluate(mu, rho=True, n_corr=True))
                el, t_el = _sync_time(lambda: gl.evaluate(mu, rho=True, n_corr=True))
                (mu_l, it_l), t_mu = _sync_time(lambda: gl.find_mu(s.n_target, 0.0, tol=1e-10))
                res.update({
                    "evaluate_direct_s": t_ed, "evaluate_lowrank_s": t_el,
                    "G_loc_rel_diff": float((el["gloc"] - ed["gloc"]).abs().max() / ed["gloc"].abs().max()),
                    "rho_rel_diff": float((el["rho"] - ed["rho"]).abs().max() / ed["rho"].abs().max()),
                    "find_mu_s": t_mu, "find_mu_evaluations": it_l})
            out[name] = res
            gd.close()
            gl.close()
    elif args.workload == "pole":
        # pseudo-Hamiltonian (pole) path against the Matsubara path, Ce-like and NiO-like
        from oracle import pole as pole_oracle
        out["config"] = "Ce-like full size; NiO-like with N_k = 1024 of its 4096 k-points"
        for name, s in _lr_pole_cases(args, synth):
            g = _context(gf, [s], "fp64")
            g.set_sigma_poles([len(s.pole.p)], s.pole.p, s.pole.V.reshape(-1), s.pole.sigma_inf.reshape(-1))
            mu = 0.3
            g.pole_occupation(mu)
            (n_p, d_p), t_occ = _sync_time(lambda: g.pole_occupation(mu))
            (mu_p, it_p), t_mu = _sync_time(lambda: g.pole_find_mu(s.n_target, 0.0, tol=1e-10))
            (_, nc_p), t_rho = _sync_time(lambda: g.pole_density_matrix(mu))
            glp, t_gl = _sync_time(lambda: g.pole_local(mu))
            eps = np.linspace(-10, 10, 2001)
            _, t_dos = _sync_time(lambda: g.pole_spectral(mu, eps, 0.05))
            g.occupation(mu)
            (n_m, d_m), t_mats = _sync_time(lambda: g.occupation(mu))
            glm = g.local(mu)
            ks = list(range(8))
            sub = pole_oracle.density(s.H[ks], s.P[ks], s.sigma_inf, s.pole.p, s.pole.V, s.beta, mu,
                                      weights=np.full(8, 1.0 / 8))
            gs = _context(gf, [synth.System(s.H[ks], s.P[ks], s.pole, s.sigma, s.beta, s.n_target)], "fp64")
            gs.set_sigma_poles([len(s.pole.p)], s.pole.p, s.pole.V.reshape(-1), s.pole.sigma_inf.reshape(-1))
            n_sub, _ = gs.pole_occupation(mu)
            gs.close()
            out[name] = {
                "n_poles": len(s.pole.p), "matrix": s.H.shape[1] + len(s.pole.p),
                "pole_occupation_s": t_occ, "matsubara_occupation_s": t_mats,
                "speedup_occupation_vs_matsubara": t_mats / t_occ,
                "pole_find_mu_s": t_mu, "pole_find_mu_evaluations": it_p,
                "pole_density_matrix_s": t_rho, "pole_local_s": t_gl, "pole_dos_2001_energies_s": t_dos,
                "N_pole_minus_matsubara": float(n_p[0] - n_m[0]),
                "G_loc_rel_diff_vs_matsubara": float((glp - glm).abs().max() / glm.abs().max()),
                "N_rel_err_vs_pole_oracle_8k": abs(n_sub[0] - sub["N"]) / sub["N"]}
            g.close()
    elif args.workload == "dmft_step":
        # the steps around the lattice sums: Lowdin projectors (Eqs. 6-7), E_imp and Delta
        # (Eqs. E^imp, dmftloop2), on the Ce-like and NiO-like (N_k = 1024) shapes
        from oracle import dmft as dmft_oracle
        out["config"] = "Ce-like full size; NiO-like generators with N_k = 1024"
        for name, s in _lr_pole_cases(args, synth):
            g = _context(gf, [s], "fp64")
            rng = np.random.default_rng(17)
            W = [np.diag(rng.uniform(0.5, 1.5, s.m)) @ p for p in s.P]
            Wp = _pack(W)
            g.set_projectors_lowdin(Wp)
            P_new, t_low = _sync_time(lambda: g.set_projectors_lowdin(Wp))
            mu = 0.3
            gl = g.local(mu)
            E, t_e = _sync_time(lambda: g.impurity_levels([1.0]))
            D, t_d = _sync_time(lambda: g.hybridization(mu, gl, [1.0]))
            ks = list(range(4))
            ref = dmft_oracle.lowdin([W[k] for k in ks])
            Pk = P_new.cpu().numpy().reshape(s.nk, s.m, -1)[ks]
            idx = [0, s.n_iw - 1]
            glh = gl.cpu().numpy().reshape(s.n_iw, s.m, s.m)
            Dr = np.array([(1j * (2 * n + 1) * np.pi / s.beta + mu) * np.eye(s.m) - E.cpu().numpy().reshape(s.m, s.m)
                           - s.sigma[n] - np.linalg.inv(glh[n]) for n in idx])
            Dg = D.cpu().numpy().reshape(s.n_iw, s.m, s.m)[idx]
            out[name] = {"lowdin_projectors_s": t_low, "impurity_levels_s": t_e, "hybridization_s": t_d,
                         "lowdin_rel_err_vs_oracle_4k": float(np.max(np.abs(Pk - np.array(ref))) /
                                                              np.max(np.abs(np.array(ref)))),
                         "delta_rel_err_vs_formula": float(np.max(np.abs(Dg - Dr)) / np.max(np.abs(Dr)))}
            g.close()
    print(json.dumps(out, default=float), flush=True)
    return 0


def main():
    args = parse()
    if args.peaks:
        return run_peaks()
    if args.workload != "ce_like" and args.impl == "ours":
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_1111_2157_gb300 import build as gfbuild
    if not gfbuild.LIB.exists():
        gfbuild.build()
    from paper_1111_2157_gb300 import gf, synth

    kw = {}
    if args.nk:
        kw["nk"] = args.nk
    if args.n_iw:
        kw["n_iw"] = args.n_iw
    s = synth.ce_like(**kw).systems[0]
    nk, nb, m, n_iw = s.nk, 40, s.m, s.n_iw
    dev = torch.device(f"cuda:{local}")
    H_d = torch.from_numpy(s.H).to(dev)
    P_d = torch.from_numpy(s.P).to(dev)
    S_d = torch.from_numpy(s.sigma).to(dev)
    Si_d = torch.from_numpy(s.sigma_inf).to(dev)
    rng = np.random.default_rng(2157)
    gbar_h = (rng.standard_normal(s.sigma.shape) + 1j * rng.standard_normal(s.sigma.shape)) * 1e-3
    gbar_d = torch.from_numpy(gbar_h).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def run_leg(precision, steps, warmup, sample_clocks, lowrank=False):
        g = gf.GreensFunction(nb, m, n_iw, s.beta, n_k=nk, device=local, precision=precision,
                              lowrank=lowrank)
        g.set_hamiltonian(H_d)
        g.set_projectors(P_d)
        g.set_sigma(S_d, Si_d)
        gloc_d = torch.empty(g.tot_sig, dtype=torch.complex128, device=dev)
        rho_d = torch.empty(g.tot_h, dtype=torch.complex128, device=dev)
        sbar_d = torch.empty(g.tot_sig, dtype=torch.complex128, device=dev)
        totals = {"launches": 0, "points": 0, "kernel_ms": 0.0, "flops": 0.0}
        passes = {name: {"kernel_ms": 0.0, "flops": 0.0, "launches": 0}
                  for name in ("find_mu", "evaluate", "backward")}
        info = {}

        def acc(name):
            st = g.stats()
            for k in totals:
                totals[k] += st[k]
            passes[name]["kernel_ms"] += st["kernel_ms"]
            passes[name]["flops"] += st["flops"]
            passes[name]["launches"] += 1

        mu_tol = MIXED_MU_TOL * s.n_target if precision == "mixed" else 1e-10

        def step():
            mu, it = g.find_mu([s.n_target], 0.0, tol=mu_tol, max_iter=60)
            acc("find_mu")
            out = g.evaluate(mu, gloc_out=gloc_d, rho_out=rho_d)
            acc("evaluate")
            g.backward(mu, gloc_bar=gbar_d, n_bar=[1.0], out=sbar_d)
            acc("backward")
            info["mu"], info["iters"], info["N"] = float(mu[0]), it, float(out["N"][0])

        for _ in range(warmup):
            step()
            flush.zero_()
        for k in totals:
            totals[k] = 0 if k in ("launches", "points") else 0.0
        for v in passes.values():
            v.update(kernel_ms=0.0, flops=0.0, launches=0)
        clocks = ClockSampler(local) if sample_clocks else None
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            step()
            if i + 1 < steps:
                flush.zero_()
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        elapsed = e0.elapsed_time(e1) / 1e3
        if ws > 1:
            t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            elapsed = float(t.item())
            torch.distributed.barrier()
        return {"g": g, "elapsed": elapsed, "totals": totals, "passes": passes, "info": info,
                "clocks": clk, "gloc": gloc_d}

    fp = run_leg(args.precision, args.steps, args.warmup, True)
    g, elapsed, totals, passes, info, clk = (fp["g"], fp["elapsed"], fp["totals"], fp["passes"],
                                             fp["info"], fp["clocks"])
    points_all = totals["points"] * ws
    value = points_all / elapsed
    achieved = totals["flops"] / (totals["kernel_ms"] / 1e3) / 1e12

    mixed = None
    if args.precision == "fp64" and not args.no_mixed:
        mx = run_leg("mixed", args.steps, args.warmup, False)
        gm = mx["g"]
        # errors of the mixed path against the FP64 GPU path at the FP64 mu*
        n_mx, _ = gm.occupation([info["mu"]])
        gl_mx = gm.local([info["mu"]])
        gl_fp = g.local([info["mu"]])
        err_n = abs(n_mx[0] - info["N"]) / abs(info["N"])
        err_g = float((gl_mx - gl_fp).abs().max() / gl_fp.abs().max())
        mt = mx["totals"]
        mixed = {"value": mt["points"] * ws / mx["elapsed"], "unit": UNIT,
                 "ms_per_step": mx["elapsed"] / args.steps * 1e3,
                 "speedup_vs_fp64_gpu": (mt["points"] / mx["elapsed"]) / (totals["points"] / elapsed),
                 "N_rel_err_vs_fp64_gpu": err_n, "G_loc_rel_err_vs_fp64_gpu": err_g,
                 "mu_star": mx["info"]["mu"],
                 "mu_tol": MIXED_MU_TOL * s.n_target,
                 "roofline": {"bound": "alu", "achieved": mt["flops"] / (mt["kernel_ms"] / 1e3) / 1e12,
                              "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": mt["flops"] / (mt["kernel_ms"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                              "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"},
                 "arithmetic": "FP32 embedding and Gauss-Jordan inverse (register tiles); FP64 Matsubara "
                               "sums, tail, k-sums and mu search; G P^+ and P G refined once with an "
                               "FP32-pair residual",
                 "kernel_choice": gm.tuning_log(), "gpu_launches": mt["launches"]}
        gm.close()
        # the FP32-pair mode (GF_PREC_PAIR, ~1e-14 of FP64), a few steps
        ps_, pw_ = min(args.steps, 3), min(args.warmup, 3)
        pl = run_leg("pair", ps_, pw_, False)
        gp = pl["g"]
        n_p, _ = gp.occupation([info["mu"]])
        pt = pl["totals"]
        mixed["pair_mode"] = {"value": pt["points"] * ws / pl["elapsed"], "unit": UNIT, "steps": ps_,
                              "ms_per_step": pl["elapsed"] / ps_ * 1e3,
                              "speedup_vs_fp64_gpu": (pt["points"] / pl["elapsed"]) / (totals["points"] / elapsed),
                              "N_rel_err_vs_fp64_gpu": abs(n_p[0] - info["N"]) / abs(info["N"]),
                              "arithmetic": "FP32 pairs (hi + lo, error-free transformations) on the FP32 "
                                            "pipes; FP64 reductions, tail and mu search",
                              "kernel_choice": gp.tuning_log()}
        gp.close()

    lowrank = None
    if args.precision == "fp64" and not args.no_mixed:
        # the same step with the eigenbasis (Woodbury) algorithm: a different algorithm, reported
        # beside the direct path's numbers, never in them
        ls_, lw_ = min(args.steps, 5), min(args.warmup, 3)
        lr = run_leg("fp64", ls_, lw_, False, lowrank=True)
        gr = lr["g"]
        n_lr, _ = gr.occupation([info["mu"]])
        gl_lr = gr.local([info["mu"]])
        gl_fp = g.local([info["mu"]])
        lt = lr["totals"]
        # and with GF_PREC_MIXED (FP32-pair band sums, FP64 m x m algebra)
        ml = run_leg("mixed", ls_, lw_, False, lowrank=True)
        gml = ml["g"]
        n_ml, _ = gml.occupation([info["mu"]])
        mlt = ml["totals"]
        mixed_lowrank = {"value": mlt["points"] * ws / ml["elapsed"], "unit": UNIT,
                         "ms_per_step": ml["elapsed"] / ls_ * 1e3, "steps": ls_,
                         "speedup_vs_direct_fp64_gpu": (mlt["points"] / ml["elapsed"]) / (totals["points"] / elapsed),
                         "N_rel_err_vs_direct": abs(n_ml[0] - info["N"]) / abs(info["N"]),
                         "gpu_launches": mlt["launches"]}
        gml.close()
        lowrank = {"value": lt["points"] * ws / lr["elapsed"], "unit": UNIT,
                   "ms_per_step": lr["elapsed"] / ls_ * 1e3, "steps": ls_,
                   "speedup_vs_direct_fp64_gpu": (lt["points"] / lr["elapsed"]) / (totals["points"] / elapsed),
                   "N_rel_err_vs_direct": abs(n_lr[0] - info["N"]) / abs(info["N"]),
                   "G_loc_rel_err_vs_direct": float((gl_lr - gl_fp).abs().max() / gl_fp.abs().max()),
                   "algorithm": "G in the eigenbasis of H_k (Woodbury identity), FP64; H_k diagonalised once",
                   "gpu_launches": lt["launches"], "mixed_precision": mixed_lowrank}
        gr.close()

    e2e = None
    if not args.no_e2e:
        # Same step through the public API with HOST buffers: inputs copied in and
        # outputs copied out inside the timed region, every step.
        H_h = torch.from_numpy(s.H).pin_memory()
        P_h = torch.from_numpy(s.P).pin_memory()
        S_h = torch.from_numpy(s.sigma).pin_memory()
        Si_h = torch.from_numpy(s.sigma_inf).pin_memory()
        gb_h = torch.from_numpy(gbar_h).pin_memory()
        gloc_h = torch.empty(g.tot_sig, dtype=torch.complex128).pin_memory()
        rho_h = torch.empty(g.tot_h, dtype=torch.complex128).pin_memory()
        sbar_h = torch.empty(g.tot_sig, dtype=torch.complex128).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        pts = 0

        def step_host():
            g.set_hamiltonian(H_h)
            g.set_projectors(P_h)
            g.set_sigma(S_h, Si_h)
            mu, _ = g.find_mu([s.n_target], 0.0, tol=1e-10, max_iter=60)
            p = g.stats()["points"]
            g.evaluate(mu, gloc_out=gloc_h, rho_out=rho_h)
            p += g.stats()["points"]
            g.backward(mu, gloc_bar=gb_h, n_bar=[1.0], out=sbar_h)
            p += g.stats()["points"]
            return p

        step_host()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pts += step_host()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([te], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            te = float(t.item())
        h2d = sum(x.numel() * x.element_size() for x in (H_h, P_h, S_h, Si_h, gb_h))
        d2h = sum(x.numel() * x.element_size() for x in (gloc_h, rho_h, sbar_h))
        e2e = {"value": pts * ws / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, _ = oracle_sample(s, info["mu"], args.cpu_seconds)
    nio = batched = None
    if rank == 0 and ws == 1 and args.precision == "fp64" and not (args.nk or args.n_iw):
        import oracle
        o = oracle.get()
        o.set_threads(cpu_cores())
        if not args.no_nio:
            nio = nio_leg(gf, synth, o)
        if not args.no_batched:
            batched = batched_leg(gf, synth, o, nk_scale=args.nk_scale)

    if args.precision == "fp64":
        peak, peak_source = FP64_PEAK_TFLOPS, "FP64 DFMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz"
    elif args.precision == "mixed":
        peak, peak_source = FP32_PEAK_TFLOPS, "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    else:
        peak, peak_source = MIXED_PEAK_TFLOPS, ("FP32 pipes: 152 SMs x 128 lanes x 2.07 GHz / 48 FP32 "
                                                "operations per FP32-pair complex multiply-add x 8 flop")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32", "pair": "f32x2"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "step": "find_mu (Newton from mu=0, tol 1e-10; mixed legs 1e-8 N_target) + fused G_loc/rho_k/N/dN/n_corr "
                               "pass + adjoint (Sigma_bar, mu_bar)",
                       "precision": args.precision, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "points_per_step": totals["points"] // args.steps,
                       "mu_evaluations_per_step": info["iters"], "mu_star": info["mu"],
                       "N_at_mu_star": info["N"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": ncu_traffic() if args.precision == "fp64" else None,
                         "kernel": {"fp64": "k_point_fp64", "mixed": "k_point_f32r (autotuned tiles)",
                                    "pair": "k_point_df64 / k_point_df64r (autotuned)"}[args.precision],
                         "peak_source": peak_source,
                         "kernel_share_of_step": totals["kernel_ms"] / 1e3 / elapsed,
                         "by_pass_tflops": {k: v["flops"] / max(v["kernel_ms"], 1e-9) / 1e9
                                            for k, v in passes.items()},
                         "by_pass_ms_per_step": {k: v["kernel_ms"] / args.steps
                                                 for k, v in passes.items()}},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": totals["launches"], "clocks": clk,
            "mixed": mixed,
            "lowrank": lowrank,
            "nio_like": nio,
            "batched": batched,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
