#!/usr/bin/env python
"""Benchmark: TU-fRG right-hand-side evaluations per second on the 24x24 / 8x8-per-cell
Rashba-Hubbard workload (N_s = 2, N_ff = 9, M = 36), split precision, plus the plain
FP64 GPU path, time-to-Lambda_c of both, the end-to-end host-buffer rate, the loop
kernel's roofline and the CPU oracle as a reported baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-flow]

One step = one full right-hand side (Fermi tables, P and C loop k-sums, Fourier
transform, projections, V.L.V) at T = 0.1 on a mid-flow state.  Inputs are resident
in HBM; the L2 is flushed (a 256 MB write) between timed steps.  N > 1 runs one
independent model instance per rank (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "rashba_hubbard_q24x24_k8x8_ff9"
METRIC = "TU-fRG RHS evals/s (split precision, <=1e-4 vertex err) on Rashba-Hubbard 24x24 q / 8x8 k per cell"
T_BENCH = 0.1
# other model configurations that --workload selects (the JSON line then names them)
WORKLOADS = {
    "rashba": (WORKLOAD, METRIC),
    "hubbard": ("hubbard_q8x8_k16x16_ff5",
                "TU-fRG RHS evals/s (split precision, <=1e-4 vertex err) on Hubbard 8x8 q / 16x16 k per cell"),
    "t2g": ("t2g_soc_q32x32_k6x6_ff9",
            "TU-fRG RHS evals/s (split precision, <=1e-4 vertex err) on t2g+SOC (N_s = 6) 32x32 q / 6x6 k per cell"),
}


class RankGroup:
    """Barrier and maximum over the ranks of one job: NCCL tensors on the GPUs, gloo on CPU tensors in the
    multi-process tests; a single process (dist None) is a group of one."""

    def __init__(self, dist=None, device="cuda"):
        self.dist, self.device = dist, device
        self.world = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(units: float, seconds: float, group: RankGroup) -> float:
    """Units processed by all ranks (each rank the same number: weak scaling) over the slowest rank's time."""
    return group.world * units / group.max(seconds)


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        load = sorted(sm)
        med = load[len(load) // 2]
        return {"sm_mhz": med, "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def tf32_peak_tflops(peaks):
    """Dense TF32 tensor peak: the measured BF16 peak times the nominal TF32 / BF16 ratio (1.1 / 2.25)."""
    return peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25


def products_tf32_flop(M, Nq):
    """3xTF32 work of one right-hand side's products: per transfer momentum and channel two complex
    M^3 GEMMs, each four real GEMMs times three TF32 products, 2 flop per multiply-add."""
    return 2.0 * 2 * 2 * 4 * 3 * float(M) ** 3 * Nq


LOOP_KERNEL_SOURCES = ("paper_1710_08830_gb300/csrc/k_loops2.cu", "paper_1710_08830_gb300/csrc/tufrg_internal.cuh")


def loop_sources_hash() -> str:
    """First 16 hex digits of the SHA-256 over every source file the two-band loop kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for rel in LOOP_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def loop_traffic_record():
    """DRAM bytes per loop-kernel launch from the committed ncu summary, if it was taken on the current sources
    (the kernel's file and the header it includes)."""
    p = os.path.join(ROOT, "profiles", "loops_traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("sources_sha256_16") != loop_sources_hash():
        return None, rec
    return rec, rec


def run_products_sweep(args):
    """Products phase per right-hand side, tensor cores (tcgen05, 3xTF32) vs CUDA cores (FP32)."""
    import numpy as np
    import torch
    from paper_1710_08830_gb300 import inputs
    from paper_1710_08830_gb300.api import PRODUCTS_SIMT, PRODUCTS_TC, SPLIT32, Model
    peaks, src = measured_peaks()
    tf32 = tf32_peak_tflops(peaks)
    rows = []
    for n_ff in (5, 9, 13):
        spec = inputs.t2g_soc(0, 0.2, 2.0, 0.4, Lq=32, nc=1, n_ff=n_ff, filling=4.0, T_mu=0.05)
        st = torch.from_numpy(inputs.random_state(spec, seed=1, scale=0.1)).cuda()
        out = torch.empty_like(st)
        row = {"n_ff": n_ff, "M": spec.M, "Nq": spec.Nq}
        for name, prod in (("tc", PRODUCTS_TC), ("simt", PRODUCTS_SIMT)):
            m = Model(spec, SPLIT32, products=prod)
            for _ in range(2):
                m.rhs(0.1, st, out=out)
            k = 5
            m.timing_begin()
            for _ in range(k):
                m.rhs(0.1, st, out=out)
            ph, _, _ = m.timing_end()
            row[f"{name}_ms"] = ph["vlv"] / k
            m.close()
        flop = products_tf32_flop(spec.M, spec.Nq)
        row["tc_tf32_tflops"] = flop / (row["tc_ms"] * 1e-3) / 1e12
        row["tc_frac_of_tf32_peak"] = row["tc_tf32_tflops"] / tf32
        row["complex_fp32_equiv_tflops_tc"] = 2.0 * 2 * 2 * 4 * float(spec.M) ** 3 * spec.Nq / (row["tc_ms"] * 1e-3) / 1e12
        rows.append(row)
    print(json.dumps({"products_sweep": rows, "tf32_peak_tflops": tf32,
                      "peak_source": f"{src} bf16 {peaks.get('bf16_tflops')} TFLOP/s x 1.1/2.25 (nominal TF32/BF16)",
                      "note": "products phase of one right-hand side (both channels, packing included), CUDA events"}))


def loops_tc_tensor_flop(n_direct, Lf, Nk, ndyh):
    """3xTF32 work of one launch of the tensor-core loop k-sum (N_s = 6): executed = MMAs as issued (128 x 112 x 8
    per instruction, 36 per stage of 4 fine-mesh rows, stages padded to 4 rows, groups of 3 momenta padded to 3);
    useful = the unpadded operands (3 dy x 36 rows, 3 momenta x 36 columns, K = 6 per fine point): per (q, k)
    2 flop x 3 TF32 passes x 4 real products x (ndyh 36) x 36 x 6."""
    groups = (n_direct + 2) // 3
    stages = (Lf + 3) // 4
    executed = float(groups) * Lf * stages * 36 * 2 * 128 * 112 * 8
    useful = float(n_direct) * Nk * 2 * 3 * 4 * (ndyh * 36) * 36 * 6
    return executed, useful


def time_rhs(m, T, state, out, k, stream, symmetric=True):
    """Mean device milliseconds of k right-hand sides (CUDA events on the model's stream), after two warm-ups."""
    import torch
    for _ in range(2):
        m.rhs(T, state, out=out, symmetric=symmetric)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        m.rhs(T, state, out=out, symmetric=symmetric)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def run_config_t2g(stream, peaks, fp32_peak, seed=0, k=10):
    """Three-orbital t2g + SOC (N_s = 6, M = 324), 32x32 q / 6x6 k per cell, split precision: RHS/s at T = 0.1 on
    the mid-flow state, the loop k-sum's roofline counted both ways (the method's complex FP32 work, and the
    3xTF32 MMA work of the tensor-core kernel), the products' roofline, and the split-vs-FP64 error."""
    import numpy as np
    import torch
    from paper_1710_08830_gb300 import inputs
    from paper_1710_08830_gb300.api import FP64, SPLIT32, Model
    spec = inputs.t2g_q32_k6_ff9(seed)
    t0 = time.perf_counter()
    m = Model(spec, SPLIT32, stream=stream)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    state, rf = m.flow(T_end=T_BENCH, stop=1e9)
    out = torch.empty_like(state)
    ms = time_rhs(m, T_BENCH, state, out, k, stream)
    m.timing_begin()
    for _ in range(3):
        m.rhs(T_BENCH, state, out=out, symmetric=True)
    ph, _, nloop = m.timing_end()
    ph = {kk: v / 3 for kk, v in ph.items()}
    loop_ms = ph["loops"] * 3 / max(1, nloop)
    ndyh = int(sum(1 for d in np.unique(spec.ff_R[:, 1][:, None] - spec.ff_R[:, 1][None, :]) if d >= 0))
    unit = spec.n_s ** 4 + spec.n_s ** 5 + ndyh * spec.n_s ** 4
    fp32_flop = 8.0 * m.n_loop_q * spec.Nk * unit
    tf32 = tf32_peak_tflops(peaks)
    loops = {"kernel": "loops_tc_kernel" if m.loops_backend == "tc" else "loops_gen_kernel",
             "backend": m.loops_backend, "avg_launch_ms": loop_ms,
             "units_per_launch": f"{m.n_loop_q} directly summed q x {spec.Nk} k",
             "method_fp32": {"unit_work": f"(N_s^4 + N_s^5 + {ndyh} N_s^4) = {unit} complex FMA per (q, k)",
                             "achieved_tflops": fp32_flop / (loop_ms * 1e-3) / 1e12, "peak_tflops": fp32_peak,
                             "frac": fp32_flop / (loop_ms * 1e-3) / 1e12 / fp32_peak,
                             "note": "the method's complex FP32 work against the FP32 FMA peak (the count used for the "
                                     "CUDA-core kernel)"}}
    if m.loops_backend == "tc":
        ex, us = loops_tc_tensor_flop(m.n_loop_q, spec.Lf, spec.Nk, ndyh)
        loops["tensor_3xtf32"] = {
            "bound": "tensor", "peak_tflops": tf32, "peak_source": "measured bf16 x 1.1/2.25 (nominal TF32/BF16)",
            "executed_tflops": ex / (loop_ms * 1e-3) / 1e12, "executed_frac": ex / (loop_ms * 1e-3) / 1e12 / tf32,
            "useful_tflops": us / (loop_ms * 1e-3) / 1e12, "useful_frac": us / (loop_ms * 1e-3) / 1e12 / tf32,
            "note": "executed counts the MMAs as issued (padded 128 x 112 tiles), useful the unpadded 108 x 108 operands; "
                    "three TF32 passes per real product, four real products per complex one"}
    n_products = m.n_loop_q if m.symmetric_state_path else spec.Nq
    prod = None
    if m.products == "tc":
        fl = products_tf32_flop(spec.M, n_products)
        prod = {"bound": "tensor", "kernel": "vlv_tc_kernel (tcgen05, 3xTF32, operands split in the kernel)", "phase_ms": ph["vlv"],
                "tf32_3pass_tflops": fl / (ph["vlv"] * 1e-3) / 1e12, "frac_tf32_3pass": fl / (ph["vlv"] * 1e-3) / 1e12 / tf32,
                "method_complex_fp32_tflops": fl / 3 / (ph["vlv"] * 1e-3) / 1e12,
                "frac_method_of_tf32_peak": fl / 3 / (ph["vlv"] * 1e-3) / 1e12 / tf32,
                "work": f"2 channels x 2 complex M^3 GEMMs per multiplied momentum ({n_products} of {spec.Nq}); the "
                        "3-pass count multiplies by the three TF32 products"}
    # accuracy: the same state through the plain FP64 path (one right-hand side)
    m64 = Model(spec, FP64, stream=stream)
    d64 = m64.rhs(T_BENCH, state).cpu().numpy()
    d32 = m.rhs(T_BENCH, state, symmetric=True).cpu().numpy()
    err = float(np.abs(d32 - d64).max() / np.abs(d64).max())
    del m64
    m.close()
    return {"workload": "t2g_soc_q32x32_k6x6_ff9", "Nq": spec.Nq, "Nk": spec.Nk, "M": spec.M, "n_s": spec.n_s,
            "rhs_per_s": 1e3 / ms, "ms_per_rhs": ms, "init_s": init_s, "T": T_BENCH,
            "phase_ms_per_rhs": ph, "roofline_loops": loops, "roofline_products": prod,
            "split_vs_fp64_maxrel": err, "products": m.products, "loops_backend": m.loops_backend,
            "products_tiles": {"width": m.products_tile_width, "tuning_ms": m.products_tiles_tuning_ms},
            "flow_to_T_steps": rf["n_steps"], "note": "state: the split flow from T0 = 10 down to T = 0.1"}


def flow_summary(r):
    return {"wall_s": r["wall_s"], "Tc": r["Tc"], "crossed": r["crossed"], "n_rhs": r["n_rhs"], "n_steps": r["n_steps"],
            "n_reject": r["n_reject"], "lead_channel": "PC"[r["lead_channel"]], "lead_q": r["lead_q"], "amax": r["amax"]}


def run_config_hubbard(stream, k=50):
    """Single-band Hubbard 8x8 q / 16x16 k per cell, N_ff = 5: split and FP64 RHS/s at T = 0.1 and the flows
    T0 = 10 -> T_end = 0.02 of both (no crossing of max|A| = 50 above T_end: a time to T_end)."""
    import numpy as np
    import torch
    from paper_1710_08830_gb300 import inputs
    from paper_1710_08830_gb300.api import FP64, SPLIT32, Model
    spec = inputs.hubbard_q8_k16_ff5()
    res = {"workload": "hubbard_q8x8_k16x16_ff5", "Nq": spec.Nq, "Nk": spec.Nk, "M": spec.M}
    states = {}
    for name, prec in (("split", SPLIT32), ("fp64", FP64)):
        t0 = time.perf_counter()
        m = Model(spec, prec, stream=stream)
        torch.cuda.synchronize()
        init_s = time.perf_counter() - t0
        st, _ = m.flow(T_end=T_BENCH, stop=1e9)
        out = torch.empty_like(st)
        ms = time_rhs(m, T_BENCH, st, out, k if name == "split" else 10, stream)
        y, r = m.flow()
        states[name] = y.cpu().numpy()
        res[name] = {"rhs_per_s": 1e3 / ms, "init_s": init_s, "flow": flow_summary(r)}
        m.close()
    res["final_state_split_vs_fp64_maxrel"] = float(np.abs(states["split"] - states["fp64"]).max() /
                                                    np.abs(states["fp64"]).max())
    res["note"] = ("time to T_end = 0.02 (max|A| stays below the stop value 50); the flows integrate the same "
                   "equations from T0 = 10 with rtol 1e-6")
    return res


def leading_form_factor(spec, state, res, stream):
    """Leading channel, momentum and form factor of a flow's last state (the survey's reading of the report): the
    eigenvector of A_X(q*) with the largest eigenvalue in modulus, its weight per irrep form factor of C4v (the
    library's tufrg_irrep_basis of the projected vertex), and the (shell, irrep) holding the most."""
    import numpy as np
    import torch
    from paper_1710_08830_gb300.api import FP64, Model
    m = Model(spec, FP64, stream=stream)
    try:
        W, lab = m.form_factors()
    except Exception:
        m.close()
        return None
    A, _ = m.project(torch.from_numpy(state).cuda())
    Ai = m.irrep_basis(A).cpu().numpy()[res["lead_channel"], res["lead_q"]]
    m.close()
    ev, vec = np.linalg.eigh(0.5 * (Ai + Ai.conj().T))
    v = vec[:, int(np.argmax(np.abs(ev)))]
    w = (np.abs(v) ** 2).reshape(spec.n_ff, spec.n_s ** 2).sum(axis=1)
    names = ("A1", "A2", "B1", "B2", "E")
    per = {}
    for i, (shell, gi, _) in enumerate(lab):
        key = f"shell {int(shell)} {names[int(gi)]}"
        per[key] = per.get(key, 0.0) + float(w[i])
    best = max(per, key=per.get)
    return {"channel": "PC"[res["lead_channel"]], "q": res["lead_q"], "form_factor": best, "weight": per[best],
            "weights": {k: round(v2, 4) for k, v2 in sorted(per.items(), key=lambda kv: -kv[1]) if v2 > 1e-3}}


def run_batch_flows(stream, n, seed=0):
    """n uneven Rashba/Hubbard flows (Lq in {16, 24, 32, 48}, N_ff in {5, 9, 13}) through tufrg_flow_batch and one by
    one, split precision; then the first crossing instance (smallest problem) again in FP64: its critical scale
    and final state against the split flow."""
    import numpy as np
    import torch
    from paper_1710_08830_gb300 import inputs
    from paper_1710_08830_gb300.api import FP64, PRODUCTS_SIMT, SPLIT32, Model, flow_batch
    specs = inputs.rashba_batch(seed=seed, n=n)
    streams = [torch.cuda.Stream() for _ in specs]
    models = [Model(sp, SPLIT32, stream=st, products=PRODUCTS_SIMT) for sp, st in zip(specs, streams)]
    torch.cuda.synchronize()
    t = time.perf_counter()
    rb = flow_batch(models)
    t_batch = time.perf_counter() - t
    del models
    seq = []
    t = time.perf_counter()
    for sp in specs:
        m = Model(sp, SPLIT32, products=PRODUCTS_SIMT)
        _, r = m.flow(want_state=False)
        seq.append(r)
        m.close()
    t_seq = time.perf_counter() - t
    same = all(a["Tc"] == b["Tc"] and a["n_steps"] == b["n_steps"] for a, b in zip(rb, seq))
    batch = {"instances": len(specs), "wall_s_batch": t_batch, "wall_s_one_by_one": t_seq,
             "flows_per_s": len(specs) / t_batch, "speedup": t_seq / t_batch,
             "rhs_total": int(sum(r["n_rhs"] for r in rb)), "crossed": int(sum(r["crossed"] for r in rb)),
             "identical_to_single_flows": same,
             "mix": {"Lq": sorted(set(sp.Lq for sp in specs)), "n_ff": sorted(set(sp.n_ff for sp in specs))}}
    crossing = None
    cand = [i for i, r in enumerate(rb) if r["crossed"]]
    if cand:
        i = min(cand, key=lambda j: specs[j].Nq * specs[j].Nk * specs[j].M)
        sp = specs[i]
        out = {}
        for name, prec in (("split", SPLIT32), ("fp64", FP64)):
            m = Model(sp, prec, stream=stream)
            y, r = m.flow()
            out[name] = (y.cpu().numpy(), r)
            m.close()
        y32, r32 = out["split"]
        y64, r64 = out["fp64"]
        lead_ff = leading_form_factor(sp, y64, r64, stream)
        # the vertex near the instability is ill-conditioned (it diverges at Lambda_c); compare the two flows also
        # at a fixed scale above it, T_end = 1.25 Lambda_c (no stop)
        above = {}
        for name, prec in (("split", SPLIT32), ("fp64", FP64)):
            m = Model(sp, prec, stream=stream)
            y, r = m.flow(T_end=1.25 * r64["Tc"], stop=1e9)
            above[name] = (y.cpu().numpy(), r)
            m.close()
        ya32, ya64 = above["split"][0], above["fp64"][0]
        crossing = {"instance": i, "Lq": sp.Lq, "n_ff": sp.n_ff, "params": {k2: round(v, 6) for k2, v in sp.params.items()}
                    if isinstance(sp.params, dict) else None,
                    "split": flow_summary(r32), "fp64": flow_summary(r64),
                    "lambda_c_ratio_split_over_fp64": r32["Tc"] / r64["Tc"],
                    "final_vertex_split_vs_fp64_maxrel": float(np.abs(y32 - y64).max() / np.abs(y64).max()),
                    "vertex_at_1p25_lambda_c_split_vs_fp64_maxrel": float(np.abs(ya32 - ya64).max() / np.abs(ya64).max()),
                    "amax_at_1p25_lambda_c": above["fp64"][1]["amax"],
                    "speedup_split_over_fp64": r64["wall_s"] / r32["wall_s"],
                    "leading_form_factor": lead_ff,
                    "note": "max|A| crosses the stop value 50: Lambda_c interpolated in ln T; final_vertex compares the last "
                            "accepted states (just past the crossing, where the vertex diverges and small differences "
                            "grow), the second error the two flows stopped at T = 1.25 Lambda_c"}
    return batch, crossing


def run_reference(args, rank, world):
    """The CPU oracle, as it stands, on bounded samples of the same workload (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1710_08830_gb300 import inputs
    spec = inputs.rashba_q24_k8_ff9(0)
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=1, scale=0.2)
    rng = np.random.default_rng(0)
    # size a step so that W + K steps take about two minutes in total
    probe = [int(x) for x in rng.choice(spec.Nq, 4, replace=False)]
    t = time.perf_counter()
    o.rhs_at(T_BENCH, st, probe, 3)
    per_q = (time.perf_counter() - t) / 4
    budget = 120.0 / max(1, args.steps + args.warmup)
    b = int(max(1, min(spec.Nq, budget / per_q)))
    units = 0.0
    for i in range(args.warmup):
        o.rhs_at(T_BENCH, st, [int(x) for x in rng.choice(spec.Nq, b, replace=False)], 3)
    t = time.perf_counter()
    for i in range(args.steps):
        o.rhs_at(T_BENCH, st, [int(x) for x in rng.choice(spec.Nq, b, replace=False)], 3)
        units += b / spec.Nq
    dt = time.perf_counter() - t
    value = units / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "Nq": spec.Nq, "Nk": spec.Nk, "M": spec.M, "T": T_BENCH,
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step: the right-hand side restricted to {b} of {spec.Nq} random transfer "
                                   f"momenta (loops, Fourier transform, projections, V.L.V); counted as {b}/{spec.Nq} RHS"},
        "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-flow", action="store_true", help="skip the time-to-Lambda_c measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile-rhs", type=int, default=0,
                    help="only evaluate this many split-precision right-hand sides on a seeded state (for ncu)")
    ap.add_argument("--profile-precision", choices=["split", "fp64"], default="split")
    ap.add_argument("--profile-symmetric-states", action="store_true",
                    help="with --profile-rhs: force the orbit-representative projections and products")
    ap.add_argument("--profile-general", action="store_true",
                    help="with --profile-rhs: the general path (projections and products at every momentum)")
    ap.add_argument("--profile-model", choices=["rashba", "t2g_q8", "t2g_q16"], default="rashba",
                    help="with --profile-rhs: the benchmark workload, or t2g + SOC at 8x8 q / 6x6 k (a small case "
                         "of the multi-orbital kernels for full profiler captures), or t2g + SOC at 16x16 q / 12x12 k "
                         "(the fine mesh of the 32x32 / 6x6 workload, Lf = 192, at a quarter of its momenta)")
    ap.add_argument("--batch-flows", type=int, default=64,
                    help="also run N uneven Rashba/Hubbard flows together (tufrg_flow_batch) and one by one, and the first "
                         "crossing instance in FP64 (0: skip)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (t2g + SOC 32x32 / 6x6, Hubbard 8x8 / 16x16) in the JSON line")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rashba",
                    help="model configuration (default: the 24x24 / 8x8 Rashba-Hubbard benchmark workload)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU path (and the accuracy check)")
    ap.add_argument("--regulator", choices=["temperature", "shell"], default="temperature",
                    help="loop regulator: the temperature flow (default) or the momentum shell of Eq. def_lmp "
                         "(flow scale Lambda, Fermi functions at T_reg = 0.05)")
    ap.add_argument("--products-sweep", action="store_true",
                    help="only time the V.L.V products (tensor cores vs CUDA cores) on t2g models with N_ff = 5, 9, 13 "
                         "(M = 180, 324, 468) at Nq = 32 x 32")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    from paper_1710_08830_gb300 import inputs
    from paper_1710_08830_gb300.api import (FP64, PRODUCTS_SIMT, SPLIT32, SYMMETRIC_STATE, SYMMETRY_AUTO, SYMMETRY_OFF,
                                            SYMMETRY_STATES, Model)

    torch.cuda.set_device(local)
    if args.products_sweep:
        run_products_sweep(args)
        return
    if args.profile_rhs > 0:
        # a short, fixed launch sequence for profilers: model set-up, then N right-hand sides
        spec = {"rashba": lambda: inputs.rashba_q24_k8_ff9(0),
                "t2g_q8": lambda: inputs.t2g_soc(0, Lq=8, nc=6, n_ff=9, filling=4.0, T_mu=0.05),
                "t2g_q16": lambda: inputs.t2g_soc(0, Lq=16, nc=12, n_ff=9, filling=4.0, T_mu=0.05)}[args.profile_model]()
        m = Model(spec, SPLIT32 if args.profile_precision == "split" else FP64,
                  symmetry=SYMMETRY_STATES if args.profile_symmetric_states else SYMMETRY_AUTO)
        st = torch.from_numpy(inputs.random_state(spec, seed=1, scale=0.2)).cuda()
        for _ in range(args.profile_rhs):
            # the timed loop's path (the values do not change the launches), or the general one
            m.rhs(T_BENCH, st, symmetric=not args.profile_general)
        torch.cuda.synchronize()
        print(json.dumps({"profile_rhs": args.profile_rhs, "workload": WORKLOAD}))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    group = RankGroup(dist, "cuda")
    barrier, allmax = group.barrier, group.max

    workload, metric = WORKLOADS[args.workload]
    if args.workload == "rashba":
        spec = inputs.rashba_q24_k8_ff9(seed=rank)     # one independent instance per rank
    elif args.workload == "hubbard":
        spec = inputs.hubbard_q8_k16_ff5()
    else:
        spec = inputs.t2g_q32_k6_ff9(seed=rank)
    if args.regulator == "shell":
        spec = spec.with_(regulator=1, T_reg=0.05)
        workload += "_shell"
        metric += " with the momentum-shell regulator (flow scale Lambda, T_reg = 0.05)"
    stream = torch.cuda.current_stream()
    t_init = time.perf_counter()
    m32 = Model(spec, SPLIT32, stream=stream)
    torch.cuda.synchronize()
    init_s = {"split": time.perf_counter() - t_init}
    t_init = time.perf_counter()
    m64 = None if args.no_fp64 else Model(spec, FP64, stream=stream)
    torch.cuda.synchronize()
    if m64 is not None:
        init_s["fp64"] = time.perf_counter() - t_init
    # a mid-flow state: the split flow from T0 = 10 down to the benchmark temperature
    state, _ = m32.flow(T_end=T_BENCH, stop=1e9)
    out = torch.empty_like(state)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        m32.rhs(T_BENCH, state, out=out, symmetric=True)
    torch.cuda.synchronize()

    # ---------------- timed region: K split-precision right-hand sides
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        m32.rhs(T_BENCH, state, out=out, symmetric=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    # per-phase breakdown and launch counts from a separate pass (phase events stay out of the timed region)
    k_phase = max(3, min(args.steps, 100))
    m32.timing_begin()
    for i in range(k_phase):
        flush.fill_(float(i))
        m32.rhs(T_BENCH, state, out=out, symmetric=True)
    phase_ms, launches, loop_launches = m32.timing_end()
    phase_ms = {k: v * args.steps / k_phase for k, v in phase_ms.items()}
    launches = launches * args.steps // k_phase
    loop_launches = loop_launches * args.steps // k_phase
    dev_ms_max = allmax(dev_ms)
    value = whole_job_rate(args.steps, dev_ms * 1e-3, group)
    ms_per_step = dev_ms_max / args.steps

    # ---------------- accuracy of the split path against the FP64 GPU path (same state)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k64 = max(3, min(args.steps, 30))
    err_split = fp64_rate = None
    if m64 is not None:
        d32 = m32.rhs(T_BENCH, state, symmetric=True).cpu().numpy()
        d64 = m64.rhs(T_BENCH, state).cpu().numpy()
        err_split = float(np.abs(d32 - d64).max() / np.abs(d64).max())

        # ---------------- plain FP64 GPU right-hand sides
        for _ in range(2):
            m64.rhs(T_BENCH, state, out=out)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k64):
            m64.rhs(T_BENCH, state, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_rate = k64 / (e0.elapsed_time(e1) * 1e-3)

    # ---------------- the same split path for a general state (projections and products at every momentum)
    for _ in range(2):
        m32.rhs(T_BENCH, state, out=out)
    torch.cuda.synchronize()
    e0.record(stream)
    kg = max(3, min(args.steps, 100))
    for _ in range(kg):
        m32.rhs(T_BENCH, state, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    general_rate = kg / (e0.elapsed_time(e1) * 1e-3)

    # ---------------- the same split path with every transfer momentum summed directly (the FP64
    # path above does not use the loop symmetries either)
    m_full = Model(spec, SPLIT32, stream=stream, symmetry=SYMMETRY_OFF)
    for _ in range(2):
        m_full.rhs(T_BENCH, state, out=out)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k64):
        m_full.rhs(T_BENCH, state, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    full_rate = k64 / (e0.elapsed_time(e1) * 1e-3)
    m_full.close()

    # ---------------- end to end through the C ABI with host buffers (pinned): every step copies its state in
    # and its dX/dT out; tufrg_rhs_host_batch overlaps the copies of neighbouring steps with the evaluations
    hs = [state.cpu().pin_memory() for _ in range(2)]
    ho = [torch.empty_like(hs[0]).pin_memory() for _ in range(2)]
    ke = max(3, min(args.steps, 100))
    m32.rhs_host_batch(T_BENCH, [hs[i % 2] for i in range(4)], [ho[i % 2] for i in range(4)], symmetric=True)
    barrier()
    t = time.perf_counter()
    m32.rhs_host_batch(T_BENCH, [hs[i % 2] for i in range(ke)], [ho[i % 2] for i in range(ke)], symmetric=True)
    e2e_rate = whole_job_rate(ke, time.perf_counter() - t, group)
    # one blocking call per step (tufrg_rhs_host), for comparison
    for _ in range(3):
        m32.rhs_host(T_BENCH, hs[0], ho[0], mask=3 | SYMMETRIC_STATE)
    t = time.perf_counter()
    for _ in range(ke):
        m32.rhs_host(T_BENCH, hs[0], ho[0], mask=3 | SYMMETRIC_STATE)
    e2e_single = whole_job_rate(ke, time.perf_counter() - t, group)
    state_bytes = int(hs[0].numel() * hs[0].element_size())

    # ---------------- band-basis exchange propagators of the benchmark state (outside the timed region)
    band = None
    if spec.n_s == 2 and spec.M <= 64:
        bout = torch.empty_like(state)
        for _ in range(3):
            m32.band_basis(state, out=bout)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nb = 20
        b0.record(stream)
        for _ in range(nb):
            m32.band_basis(state, out=bout)
        b1.record(stream)
        torch.cuda.synchronize()
        band = {"ms": b0.elapsed_time(b1) / nb, "precision": "FP32 (split model)",
                "note": "tufrg_band_basis: transformation matrices U(s), X(u) by a k-sum over the fine mesh, then "
                        "U^dagger P U and X^dagger C X for every momentum (Sec. 3.4)"}

    # ---------------- time-to-Lambda_c (full flows from T0 = 10)
    flows = None
    if not args.no_flow:
        def summary(r):
            return {"wall_s": r["wall_s"], "Tc": r["Tc"], "crossed": r["crossed"], "n_rhs": r["n_rhs"],
                    "n_steps": r["n_steps"], "lead_channel": "PC"[r["lead_channel"]], "lead_q": r["lead_q"],
                    "amax": r["amax"]}
        _, r32 = m32.flow()
        flows = {"split": summary(r32), "init_s": init_s,
                 "note": "Tc is the crossing of max|A| = 50 when crossed == 1, else the end temperature 0.02 (a time to "
                         "T_end); init_s is the model set-up (eigensystem, tables, autotuning), not part of wall_s"}
        if m64 is not None:
            _, r64 = m64.flow()
            flows["fp64"] = summary(r64)
    batch = crossing = None
    if args.batch_flows > 0 and args.workload == "rashba":
        batch, crossing = run_batch_flows(stream, args.batch_flows, seed=rank)
    configs = None
    if not args.no_configs and args.workload == "rashba":
        peaks0, _ = measured_peaks()
        props0 = torch.cuda.get_device_properties(local)
        fp32_peak0 = props0.multi_processor_count * 128 * 2 * peaks0.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        configs = {"t2g": run_config_t2g(stream, peaks0, fp32_peak0, seed=rank), "hubbard": run_config_hubbard(stream)}
    clocks = sampler.stop()

    # ---------------- roofline of the dominant kernel (the loop k-sum)
    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    sm_max = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    ns = spec.n_s
    ndy_half = int(sum(1 for d in np.unique(spec.ff_R[:, 1][:, None] - spec.ff_R[:, 1][None, :]) if d >= 0))
    unit_cfma = ns ** 4 + ns ** 5 + ndy_half * ns ** 4
    # one launch sums every fine k for each directly evaluated transfer momentum (the loop symmetries
    # supply the other momenta)
    flops_per_launch = 8.0 * m32.n_loop_q * spec.Nk * unit_cfma
    # the timed loop's products run at the orbit representatives when the state symmetries hold
    n_products = m32.n_loop_q if m32.symmetric_state_path else spec.Nq
    loop_ms_avg = phase_ms["loops"] / max(1, loop_launches)
    achieved = flops_per_launch / (loop_ms_avg * 1e-3) / 1e12
    trec = loop_traffic_record()[0] if args.workload == "rashba" else None   # recorded for that workload
    kname = ("loops2_kernel (split-precision two-band loop k-sum)" if spec.n_s == 2
             else "loops_gen_kernel (split-precision multi-orbital loop k-sum)")
    roofline = {"bound": "alu", "kernel": kname,
                "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops,
                "traffic": (trec["dram_bytes_per_launch"] if trec else None),
                "peak_source": f"FP32 FMA peak derived: {sm_count} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz",
                "algorithmic_flops_per_launch": flops_per_launch,
                "unit_work": f"(N_s^4 + N_s^5 + {ndy_half} N_s^4) = {unit_cfma} complex FMA per (q, k) pair",
                "units_per_launch": f"{m32.n_loop_q} directly summed q x {spec.Nk} k",
                "avg_launch_ms": loop_ms_avg}
    if m32.loops_backend == "tc":
        # the tensor-core loop kernel: its bound is the TF32 tensor pipe; the method's FP32 count stays beside it
        ex, us = loops_tc_tensor_flop(m32.n_loop_q, spec.Lf, spec.Nk, ndy_half)
        tf32 = tf32_peak_tflops(peaks)
        roofline = {"bound": "tensor", "kernel": "loops_tc_kernel (tcgen05 3xTF32 loop k-sum, N_s = 6)",
                    "achieved": ex / (loop_ms_avg * 1e-3) / 1e12, "peak": tf32, "unit": "TFLOP/s",
                    "frac": ex / (loop_ms_avg * 1e-3) / 1e12 / tf32, "traffic": None,
                    "peak_source": "measured bf16 x 1.1/2.25 (nominal TF32/BF16)",
                    "algorithmic_flops_per_launch": ex,
                    "unit_work": "36 MMAs of 128 x 112 x 8 (TF32) per stage of 4 fine-mesh rows, per column and "
                                 "group of 3 momenta",
                    "units_per_launch": f"{m32.n_loop_q} directly summed q x {spec.Nk} k",
                    "useful_frac": us / (loop_ms_avg * 1e-3) / 1e12 / tf32,
                    "method_fp32": {"achieved": achieved, "peak": fp32_peak_tflops, "frac": achieved / fp32_peak_tflops,
                                    "unit_work": f"(N_s^4 + N_s^5 + {ndy_half} N_s^4) = {unit_cfma} complex FMA per (q, k)"},
                    "avg_launch_ms": loop_ms_avg}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        o = oracle.Oracle(spec)
        st_np = state.cpu().numpy()
        o.rhs(T_BENCH, st_np, 3)   # warm
        t = time.perf_counter()
        n_cpu = 2
        for _ in range(n_cpu):
            o.rhs(T_BENCH, st_np, 3)
        cpu_rate = n_cpu / (time.perf_counter() - t)
        cpu = {"value": cpu_rate, "unit": "RHS/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{n_cpu} full right-hand sides of the same workload (after one warm-up)"}

    if rank == 0:
        line = {
            "metric": metric, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload, "Lq": spec.Lq, "nc": spec.nc, "Nq": spec.Nq, "Nk": spec.Nk,
                       "n_s": spec.n_s, "n_ff": spec.n_ff, "M": spec.M, "T": T_BENCH, "regulator": args.regulator,
                       "precision": "split (FP32 loop sums, FP64 state)",
                       "products": m32.products, "products_tuning_ms": m32.products_tuning_ms,
                       "loop_momenta_summed": m32.n_loop_q, "symmetric_state": True,
                       "loop_tiles": {"ky_chunks": m32.loop_ky_chunks, "tuning_ms": m32.loop_tiles_tuning_ms},
                       "products_tiles": {"width": m32.products_tile_width, "tuning_ms": m32.products_tiles_tuning_ms},
                       "symmetric_state_path": m32.symmetric_state_path,
                       "symmetric_state_tuning_ms": m32.symmetric_state_tuning_ms,
                       "l2": "flushed (256 MB write) between timed steps", "instances": f"{world} (seed = rank)"},
            "split_vs_fp64_maxrel": err_split,
            "fp64_gpu": ({"value": fp64_rate, "unit": "RHS/s", "speedup_split": value / world / fp64_rate,
                          "note": "every transfer momentum summed directly"} if fp64_rate else None),
            "rhs_general_state": {"value": general_rate, "unit": "RHS/s",
                                  "note": "tufrg_rhs without TUFRG_SYMMETRIC_STATE: projections and products at every "
                                          "momentum (the timed loop evaluates the flow state, which has the symmetries)"},
            "split_every_q_summed": {"value": full_rate, "unit": "RHS/s",
                                     "note": "split path with the loop symmetries off (same loop work as fp64_gpu)"},
            "time_to_lambda_c": flows,
            "phase_ms_per_rhs": {k: v / args.steps for k, v in phase_ms.items()},
            "gpu_launches": launches,
            "e2e": {"value": e2e_rate, "unit": "RHS/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes, "api": "tufrg_rhs_host_batch (copies of neighbouring steps "
                    "overlapped with the evaluations)", "one_call_per_step": e2e_single},
            "roofline": roofline,
            "roofline_products": ({"bound": "tensor", "kernel": "vlv_tc_kernel (tcgen05, 3xTF32, operands split in the kernel)",
                                   "achieved": products_tf32_flop(spec.M, n_products) / (phase_ms["vlv"] / args.steps * 1e-3) / 1e12,
                                   "peak": tf32_peak_tflops(peaks), "unit": "TFLOP/s",
                                   "frac": products_tf32_flop(spec.M, n_products) / (phase_ms["vlv"] / args.steps * 1e-3) / 1e12
                                           / tf32_peak_tflops(peaks),
                                   "peak_source": "measured bf16 x 1.1/2.25 (nominal TF32/BF16)",
                                   "work": f"2 channels x 2 complex M^3 GEMMs x 4 real x 3 TF32 per multiplied momentum "
                                           f"({n_products} of {spec.Nq}); the phase time includes the symmetric scatter"}
                                  if m32.products == "tc" else None),
            "cpu_baseline": cpu,
            "batch_flows": batch,
            "flow_to_lambda_c": crossing,
            "other_configs": configs,
            "band_basis": band,
            "clocks": clocks,
            "peaks_source": peak_src,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
