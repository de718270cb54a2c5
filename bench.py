#!/usr/bin/env python
"""Throughput of the TTN-HEOM hot path on GB300.

One step = one full ps1 step (Phi_{dt/2} then Phi*_{dt/2}: every node and bond
flow with RK4, every QR gauge move and environment update) of the 7-site
Frenkel exciton chain: 21 Drude/Pade features, Fock depth 8, balanced binary
tree, bond rank 20, FP64, dt = 0.05 fs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas of the
same propagation (a single TTN sweep has no data-parallel split), launched one
process per GPU by torch.distributed.run; value = all steps of all ranks / the
slowest rank's time.

Beside the headline the line carries:
- the mixed form (FP32 contractions) of the same workload;
- the same chain at bond rank 64 in both forms;
- 256 uneven spin-boson instances batched, in both forms;
- the end-to-end rate through the API;
- the roofline of the dominant kernel class;
- the FP64 CPU oracle as cpu_baseline.

--rank64-only and --accuracy-steps print only the rank-64 leg or a long rho_S
trajectory comparison instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "HEOM-TTN steps/s & node-contraction TFLOP/s vs plain FP64 at RDM err <=1e-6"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (152 SMs x 2 FP64 FMA/clk/SM x ~2.07 GHz)
WORKLOAD = "7-site Frenkel exciton chain, 21 features (1 Drude + 2 Pade per site), depth 8, BTT, rank 20, ps1, dt 0.05 fs"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
APPLY_DRAM_BYTES = 237703   # ncu: mean DRAM bytes (read + write) per k_apply launch of one timed step


def workload():
    return W.exciton_chain(n_steps=5000)


# ----------------------------------------------------------------------------
# CPU oracle leg (runs in a separate single-threaded process)
# ----------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import ttn
w = W.exciton_chain(n_steps=5000)
budget, max_steps = {budget}, {max_steps}
st = ttn.from_workload(w)
rhos, t0, n = [], time.perf_counter(), 0
while n < max_steps:
    st.step(w.dt, "ps1")
    n += 1
    rhos.append(st.rdm().reshape(-1).tolist())
    if time.perf_counter() - t0 > budget:
        break
el = time.perf_counter() - t0
print(json.dumps({{"steps": n, "seconds": el, "rho": [[[z.real, z.imag] for z in r] for r in rhos]}}))
"""


def run_oracle(budget_s: float, max_steps: int, threads: int = 1) -> dict:
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, budget=budget_s, max_steps=max_steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle subprocess failed:\n" + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["rho"] = [np.array([complex(a, b) for a, b in row]).reshape(7, 7) for row in out["rho"]]
    return out


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------
def replica_max(x: float, dist, device) -> float:
    """The largest per-rank value over the ranks (the slowest replica's time);
    x itself when there is no process group."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world: int, steps: int, ms_max: float) -> float:
    """Whole-job steps/s of `world` replicas that each ran `steps` steps, timed
    by the slowest one."""
    return world * steps / (ms_max * 1e-3)


def make_gpu(pkg, w, device, precision=0):
    return pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0,
                          drives=w.drives, device=device, precision=precision)


def timed_steps(torch, g, w, K, flush):
    """K single steps, each bracketed by CUDA events on the library's stream,
    with an L2 flush (write of 256 MB) between them outside the events."""
    total = 0.0
    stream = g.stream
    for _ in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.ttn_step(w.dt, 1, 1)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    return total  # ms


def rank64_leg(args, pkg, torch, flush, local_rank, forms=(("fp64", 0), ("mixed_fp32", 1))):
    """The 7-site chain at bond rank 64 in the FP64 and mixed forms: steps/s,
    per-class kernel time and the mixed-vs-FP64 RDM difference."""
    w64 = W.exciton_chain(rank=64)
    k64 = max(2, min(args.steps, 5))
    res = {}
    rhos = {}
    for label, prec in forms:
        gg = make_gpu(pkg, w64, local_rank, precision=prec)
        if prec == pkg.TTN_MIXED_FP32 and args.tensor_cores is not None:
            gg.ttn_set_params(tensor_cores=args.tensor_cores)
        if not args.no_autotune:
            gg.ttn_autotune(2)
        gg.ttn_step(w64.dt, 1, 1)  # warm-up (graph capture)
        torch.cuda.synchronize()
        gg.ttn_stats_reset()
        ms64 = timed_steps(torch, gg, w64, k64, flush)
        fl64 = gg.ttn_stats(0)[1]
        gg.ttn_stats_reset()
        gg.ttn_profile(True)
        timed_steps(torch, gg, w64, 1, flush)
        gg.ttn_profile(False)
        pr = {k: (gg.ttn_stats(k)[1], gg.ttn_profile_read(k)) for k in range(4)}
        rhos[label] = gg.ttn_rdm()
        res[label] = {"steps_per_s": k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64,
                      "node_contraction_gflop_per_step": fl64 / k64 / 1e9,
                      "node_contraction_tflops_kernel": pr[0][0] / (pr[0][1] * 1e-3) / 1e12 if pr[0][1] > 0 else None,
                      "kernel_ms_per_step": {n_: pr[k][1] for k, n_ in
                                             enumerate(("k_apply", "environment", "qr", "other"))}}
        gg.close()
    out = {"workload": "7-site exciton chain as above at bond rank 64 (state 1.97 M complex, nodes 64x64x64)",
           "steps_timed": k64, **res}
    if "fp64" in res and "mixed_fp32" in res:
        out["mixed_speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res["mixed_fp32"]["ms_per_step"]
        out["rdm_max_abs_mixed_vs_fp64_gpu"] = float(np.max(np.abs(rhos["fp64"] - rhos["mixed_fp32"])))
        out["steps_compared"] = 1 + k64 + 1
    return out


def accuracy_leg(args, pkg, torch, w, local_rank):
    """rho_S of the mixed form against the FP64 form over a long trajectory of
    the bench workload: max-abs difference over all steps, at the end, and the
    trace drift of each form."""
    ga = make_gpu(pkg, w, local_rank)
    if args.accuracy_vs == "mixed":
        gb = make_gpu(pkg, w, local_rank, precision=pkg.TTN_MIXED_FP32)
    else:  # FP64 again, with another summation order (no CTA split of the contractions)
        gb = make_gpu(pkg, w, local_rank)
        gb.ttn_set_params(max_split=1)
    t0 = np.trace(ga.ttn_rdm()).real
    worst, worst_step = 0.0, 0
    trail = []  # (step, max-abs difference) at about 20 points along the run
    every_trail = max(1, args.accuracy_steps // 20)
    for k in range(args.accuracy_steps):
        ga.ttn_step(w.dt, 1, 1)
        gb.ttn_step(w.dt, 1, 1)
        if (k + 1) % args.accuracy_every == 0 or k + 1 == args.accuracy_steps:
            ra, rb = ga.ttn_rdm(), gb.ttn_rdm()
            e = float(np.max(np.abs(ra - rb)))
            if e > worst:
                worst, worst_step = e, k + 1
            if (k + 1) % every_trail == 0:
                trail.append([k + 1, e, float(np.max(np.abs(ra)))])
    out = {"workload": WORKLOAD, "steps": args.accuracy_steps, "compared_every": args.accuracy_every,
           "compared": "FP64 vs " + ("mixed FP32" if args.accuracy_vs == "mixed" else "FP64 with another summation order"),
           "rdm_max_abs_diff": worst, "at_step": worst_step,
           "rdm_max_abs_at_end": float(np.max(np.abs(ra - rb))),
           "trace_drift_fp64": float(abs(np.trace(ra).real - t0)),
           "trace_drift_second": float(abs(np.trace(rb).real - t0)),
           "trail_step_err_maxabsrho": trail}
    ga.close()
    gb.close()
    return out


def measure_peaks(torch, dev) -> dict:
    """Dense matmul rates of this GPU measured in this run (torch.matmul, CUDA
    events, best of `reps` after one warm-up): FP64 (4096^3), FP32 on the CUDA
    cores (TF32 off, 8192^3), TF32 tensor cores (8192^3) and BF16 (8192^3),
    2 n^3 FLOP per product. They are the roofline denominators of the pipes the
    kernels use (FP64: the node contractions of the FP64 form; FP32: the mixed
    form on the CUDA cores; TF32: its tensor-core contractions)."""
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dtype, n, tf32, reps in (("fp64", torch.float64, 4096, False, 5),
                                          ("fp32_simt", torch.float32, 8192, False, 5),
                                          ("tf32", torch.float32, 8192, True, 10),
                                          ("bf16", torch.bfloat16, 8192, False, 10)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device=dev).to(dtype)
            b = torch.randn(n, n, device=dev).to(dtype)
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name + "_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    out["how"] = "torch.matmul best of 5-10 (CUDA events) in this run: FP64 4096^3, FP32 (TF32 off) / TF32 / BF16 8192^3"
    return out


def config1_leg(pkg, torch, local_rank, flush) -> dict:
    """Spin-boson tensor train (H = 0.5 sz + sx, Drude lambda 0.5, omega_c 1,
    beta 1, 1 Drude + 3 Pade features, depth 10, rank 10, dt 0.01), 1000 ps1
    steps in FP64: steps/s of the graph-replayed step and rho_S against the
    stored oracle trajectory (every 10th step)."""
    w = W.spin_boson_tt(n_steps=1000)
    rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", "spin_boson_tt_k4_n10_r10.txt"))
    g = make_gpu(pkg, w, local_rank)
    err = float(np.max(np.abs(g.ttn_rdm().reshape(-1) - (rows[0, 1::2] + 1j * rows[0, 2::2]))))
    for r in rows[1:]:
        g.ttn_step(w.dt, 1, int(r[0]) - int(round(g.ttn_time() / w.dt)))
        err = max(err, float(np.max(np.abs(g.ttn_rdm().reshape(-1) - (r[1::2] + 1j * r[2::2])))))
    g.close()
    g = make_gpu(pkg, w, local_rank)
    g.ttn_step(w.dt, 1, 3)
    torch.cuda.synchronize()
    with torch.cuda.stream(g.stream):
        flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(g.stream)
    g.ttn_step(w.dt, 1, 1000)
    b.record(g.stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    g.close()
    return {"workload": "spin-boson tensor train: K = 4 (1 Drude + 3 Pade), depth 10, rank 10, 4 nodes, ps1 FP64, "
                        "dt 0.01, 1000 steps", "steps_per_s": 1000 / (ms * 1e-3), "ms_per_step": ms / 1000,
            "rdm_max_abs_vs_stored_oracle": err, "steps_compared": int(rows[-1, 0]),
            "l2": "state L2-resident (39 kB): one flush before the 1000 steps"}


def ps2_leg(args, pkg, torch, local_rank) -> dict:
    """Adaptive rank (ps2) on the driven two-level system with the structured
    bath (Drude + three Brownian peaks + Pade features, depth 10, binary tree,
    ps2_atol 1e-6, ratio 2), the plain SVD rule against the learned rank
    proposer. The network is trained on the GPU (the library's forward,
    backward and Adam kernels) on the split records of rule runs of two other
    bath sizes, then both forms run the same window."""
    cap, npd, n = args.ps2_cap, args.ps2_pade, args.ps2_steps
    leg_t0 = time.perf_counter()

    def run(w, net=None, record=False, steps=None):
        nn = n if steps is None else steps
        g = pkg.from_model(w.H, w.baths, w.depth, w.parent, w.leg_node, w.ranks, rho0=w.rho0, drives=w.drives,
                           params={"max_rank": cap, "ps2_atol": w.ps2_atol}, device=local_rank)
        if net is not None:
            g.ttn_set_rank_proposer(net)
        g.ttn_stats_reset()
        rhos, ranks = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(nn):
            g.ttn_step(w.dt, pkg.TTN_PS2, 1)
            rhos.append(g.ttn_rdm())
            if record and (k + 1) % max(1, nn // 10) == 0:
                ranks.append([k + 1, int(max(g.ttn_get_ranks()))])
        el = time.perf_counter() - t0
        prop = g.ttn_proposer_stats()
        fl = g.ttn_stats(2)[1]
        return g, np.array(rhos), el, ranks, prop, fl

    # training records from rule runs of other bath sizes (same family)
    feats, labels = [], []
    n_train = min(n, 40)
    for tp in (max(0, npd - 2), npd + 1):
        wt = W.driven_structured_tls(n_pade=tp, depth=10, cap=cap)
        g, _, _, _, _, _ = run(wt, steps=n_train)
        f, y = g.ttn_split_log()
        feats.append(f)
        labels.append(y)
        g.close()
    feats, labels = np.concatenate(feats), np.concatenate(labels)
    net = pkg.RankProposer(seed=1, device=local_rank)
    t0 = time.perf_counter()
    hist = net.train(feats, labels, steps=400, lr=3e-3)
    train_s = time.perf_counter() - t0
    acc = float(np.mean(net.forward(feats).argmax(1).cpu().numpy() == labels))

    w = W.driven_structured_tls(n_pade=npd, depth=10, cap=cap)
    g0, r0, el0, ranks0, _, fl0 = run(w, record=True)
    n_splits = len(g0.ttn_split_log()[1])
    g1, r1, el1, ranks1, (proposed, accepted), fl1 = run(w, net, record=True)
    g0.close()
    g1.close()
    return {"workload": f"driven TLS, structured bath: K = {w.K} (1 Drude + 6 Brownian + {npd} Pade), depth 10, "
                        f"binary tree ({len(w.parent)} nodes), ps2 atol 1e-6 ratio 2 cap {cap}, dt 0.01, {n} steps",
            "svd_rule": {"steps_per_s": n / el0, "qr_svd_gflop": fl0 / 1e9, "splits": n_splits,
                         "max_rank_trajectory": ranks0},
            "learned": {"steps_per_s": n / el1, "qr_svd_gflop": fl1 / 1e9, "splits_proposed": proposed,
                        "splits_accepted": accepted,
                        "fraction_skipping_full_svd": accepted / proposed if proposed else 0.0,
                        "max_rank_trajectory": ranks1,
                        "training": {"records": int(len(labels)), "steps": 400, "loss_first_last": [hist[0], hist[-1]],
                                     "train_accuracy": acc, "seconds": train_s,
                                     "source": f"rule runs of the same family with {max(0, npd - 2)} and {npd + 1} "
                                               f"Pade features, {n_train} steps each"}},
            "speedup_learned_vs_rule": el0 / el1,
            "rdm_max_abs_learned_vs_rule": float(np.max(np.abs(r1 - r0))),
            "timing": "host wall clock (ps2 synchronises at every split)",
            "leg_seconds": time.perf_counter() - leg_t0}


def paper_models_leg(pkg, torch, local_rank, flush, sweeps: bool) -> dict:
    """The paper's example models (Sec. 3.2 Table 1, Sec. 3.4, Sec. 3.2.3 Table 2)
    on the GPU: steps/s of the structured spin-boson (1000 fs) and of the
    three-site FMO model with six Brownian peaks at 77 K (45 features), and --
    with `sweeps` -- the convergence study of Table 2: the time-averaged
    |rho_11 - rho_11^ref| over 1000 fs for hierarchy depths (panel a, BTT,
    reference depth 25) and bond ranks (panels b / c, BTT and TT, reference
    rank 40)."""
    def timed(w, steps, precision=0):
        g = make_gpu(pkg, w, local_rank, precision=precision)
        g.ttn_step(w.dt, 1, 2)
        torch.cuda.synchronize()
        with torch.cuda.stream(g.stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        g.ttn_step(w.dt, 1, steps)
        b.record(g.stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        rho = g.ttn_rdm()
        g.close()
        return steps / (ms * 1e-3), rho

    def traj(w, steps):
        g = make_gpu(pkg, w, local_rank)
        out = []
        for _ in range(steps):
            g.ttn_step(w.dt, 1, 1)
            out.append(g.ttn_rdm()[1, 1].real)  # rho_11 of the paper = the second state's population
        g.close()
        return np.array(out)

    res = {}
    # ML-MCTDH on the same machinery (Sec. 3.2.4): the thermofield star bath of the listing
    from paper_2603_17711_gb300 import mctdh
    sb = W.star_boson_mctdh()
    fr, gs = mctdh.thermofield_modes(sb.bo, sb.beta, sb.cutoff, sb.n_modes)
    g = pkg.TTN(sb.parent, sb.leg_node, sb.leg_dims, sb.ranks)
    g.sop_load(mctdh.mctdh_sop(sb.H, sb.Q, fr, gs, sb.dim))
    g.bind(local_rank)
    r0 = np.zeros((2, 2), np.complex128)
    r0[:, 0] = sb.psi0
    g.ttn_set_rdo0(r0)
    g.ttn_step(sb.dt, 1, 2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(g.stream)
    g.ttn_step(sb.dt, 1, sb.n_steps)
    b.record(g.stream)
    b.synchronize()
    rho = mctdh.rho_from_root(g.ttn_get_node(0).reshape(2, 2, -1))
    g.close()
    res["mctdh_star_boson"] = {"workload": sb.name + ", ps1, dt 1 fs, 200 steps", "steps_per_s":
                               sb.n_steps / (a.elapsed_time(b) * 1e-3), "population_1_at_202_fs": float(rho[1, 1].real)}
    w = W.structured_spin_boson()
    sps, rho = timed(w, 1000)
    res["structured_spin_boson"] = {"workload": w.name + ", dt 1 fs, 1000 steps, ps1 FP64", "steps_per_s": sps,
                                    "rho_11_at_1000_fs": float(rho[1, 1].real)}
    w = W.fmo3(T=77.0)
    s64, r64 = timed(w, 200)
    s32, r32 = timed(w, 200, precision=pkg.TTN_MIXED_FP32)
    res["fmo3_77K_bo6"] = {"workload": w.name + ", dt 0.05 fs, 200 steps after 2 warm-up steps, ps1",
                           "steps_per_s_fp64": s64, "steps_per_s_mixed": s32,
                           "rdm_max_abs_mixed_vs_fp64": float(np.max(np.abs(r64 - r32))),
                           "populations_fp64": [float(r64[i, i].real) for i in range(3)]}
    if sweeps:
        n = 1000
        ref_a = traj(W.convergence_spin_boson("a", depth=25, rank=40), n)
        res["table2_depth_sweep_btt"] = {
            str(d): float(np.mean(np.abs(traj(W.convergence_spin_boson("a", depth=d, rank=40), n) - ref_a)))
            for d in (2, 4, 6, 10, 14)}
        for tree in ("btt", "tt"):
            ref = traj(W.convergence_spin_boson("b", depth=25, rank=40, tree=tree), n)
            res[f"table2_rank_sweep_{tree}"] = {
                str(r): float(np.mean(np.abs(traj(W.convergence_spin_boson("b", depth=25, rank=r, tree=tree), n) - ref)))
                for r in (2, 4, 8, 12, 16, 24, 32)}
        res["table2_note"] = ("mean over 1000 steps (1 fs) of |rho_11 - rho_11(reference)|; panel a: depth sweep "
                              "against depth 25 (BTT, rank 40); panels b, c: rank sweep against rank 40 at depth 25")
    return res


def vmf_leg(pkg, torch, local_rank) -> dict:
    """Direct integration (vmf, dopri5 with ode_rtol 1e-5 / ode_atol 1e-7) of the
    7-site chain at rank 20 after 20 ps1 steps, against ps1 continued over the
    same 20 steps, and the mix strategy (ps2 then vmf) on the adaptive-rank
    workload."""
    w = W.exciton_chain()
    ga, gb = make_gpu(pkg, w, local_rank), make_gpu(pkg, w, local_rank)
    ga.ttn_step(w.dt, 1, 20)
    gb.ttn_step(w.dt, 1, 20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ga.ttn_step(w.dt, pkg.TTN_VMF, 20)
    ra = ga.ttn_rdm()
    el = time.perf_counter() - t0
    gb.ttn_step(w.dt, 1, 20)
    rb = gb.ttn_rdm()
    ga.close()
    gb.close()
    out = {"workload": "7-site chain at rank 20 (as the headline), 20 vmf steps after 20 ps1 steps",
           "steps_per_s": 20 / el, "rdm_max_abs_vmf_vs_ps1": float(np.max(np.abs(ra - rb))),
           "timing": "host wall clock (the step control synchronises)"}
    wm = W.driven_structured_tls(n_pade=1, depth=10, cap=16)
    g = pkg.from_model(wm.H, wm.baths, wm.depth, wm.parent, wm.leg_node, wm.ranks, rho0=wm.rho0, drives=wm.drives,
                       device=local_rank, params={"max_rank": 16, "ps2_atol": 1e-6})
    t0 = time.perf_counter()
    g.ttn_step(wm.dt, pkg.TTN_MIX, 40)
    g.ttn_rdm()
    out["mix"] = {"workload": "driven TLS, structured bath, K = 8, depth 10, ps2 (atol 1e-6, cap 16) then vmf, 40 steps",
                  "steps_per_s": 40 / (time.perf_counter() - t0), "ranks_at_end": [int(x) for x in g.ttn_get_ranks()]}
    g.close()
    return out


def bench_ours(args, rank, world, local_rank):
    import torch
    import paper_2603_17711_gb300 as pkg
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = workload()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if args.accuracy_steps:  # long trajectory: mixed against FP64 on the GPU, step by step
        if rank == 0:
            print(json.dumps({"accuracy": accuracy_leg(args, pkg, torch, w, local_rank)}), flush=True)
        return
    if args.paper_only:  # the paper's example models with the Table 2 convergence sweeps
        if rank == 0:
            print(json.dumps({"paper_models": paper_models_leg(pkg, torch, local_rank, flush, True)}), flush=True)
        return
    if args.ps2_only:  # only the adaptive-rank leg
        if rank == 0:
            print(json.dumps({"ps2_learned_rank": ps2_leg(args, pkg, torch, local_rank)}), flush=True)
        return
    if args.rank64_only:  # profiling aid: only the rank-64 leg, in the form asked for
        forms = (("fp64", 0),) if args.rank64_only == "fp64" else (("mixed_fp32", pkg.TTN_MIXED_FP32),)
        if rank == 0:
            print(json.dumps({"precision_rank64": rank64_leg(args, pkg, torch, flush, local_rank, forms)}), flush=True)
        return

    # ---- device-timed steps (value) ----
    g = make_gpu(pkg, w, local_rank)
    tune_s = None
    if not args.no_autotune:  # launch shapes picked by measurement, before any timed step
        t0 = time.perf_counter()
        g.ttn_autotune(3)
        tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        g.ttn_step(w.dt, 1, 1)
    torch.cuda.synchronize()
    g.ttn_stats_reset()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        wall0 = time.perf_counter()
        ms = timed_steps(torch, g, w, args.steps, flush)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = sum(g.ttn_stats(k)[0] for k in range(4))
    flops = {k: g.ttn_stats(k)[1] for k in range(4)}
    ms_max = replica_max(ms, dist, dev)

    # ---- per-kernel-class device time (roofline of the dominant kernel), taken
    # from event-record nodes inside the same replayed step graph ----
    g.ttn_stats_reset()
    g.ttn_profile(2)
    ms_prof = timed_steps(torch, g, w, args.steps, flush)
    g.ttn_profile(False)
    prof = {k: (g.ttn_stats(k)[0], g.ttn_stats(k)[1], g.ttn_profile_read(k)) for k in range(4)}
    rho_gpu_final = g.ttn_rdm()
    g.close()

    # ---- mixed-precision form on the same workload (FP32 contractions) ----
    gm = make_gpu(pkg, w, local_rank, precision=pkg.TTN_MIXED_FP32)
    if not args.no_autotune:
        gm.ttn_autotune(3)
    for _ in range(args.warmup):
        gm.ttn_step(w.dt, 1, 1)
    torch.cuda.synchronize()
    gm.ttn_stats_reset()
    ms_mixed = timed_steps(torch, gm, w, args.steps, flush)
    mixed_flops = gm.ttn_stats(0)[1]
    gm.ttn_stats_reset()
    gm.ttn_profile(2)
    timed_steps(torch, gm, w, args.steps, flush)
    gm.ttn_profile(False)
    prof_m = {k: (gm.ttn_stats(k)[0], gm.ttn_stats(k)[1], gm.ttn_profile_read(k)) for k in range(4)}
    gm.close()
    # accuracy of the mixed form against the FP64 form over the same steps
    ga = make_gpu(pkg, w, local_rank)
    gb = make_gpu(pkg, w, local_rank, precision=pkg.TTN_MIXED_FP32)
    mixed_err = 0.0
    n_cmp = args.warmup + 2 * args.steps
    for _ in range(n_cmp):
        ga.ttn_step(w.dt, 1, 1)
        gb.ttn_step(w.dt, 1, 1)
        mixed_err = max(mixed_err, float(np.max(np.abs(ga.ttn_rdm() - gb.ttn_rdm()))))
    ga.close()
    gb.close()

    # ---- precision workload: the same chain at bond rank 64 (QRs up to 4096 x 64) ----
    r64 = None if args.no_rank64 else rank64_leg(args, pkg, torch, flush, local_rank)
    # ---- the spin-boson tensor train, 1000 steps against the stored oracle trajectory ----
    c1 = config1_leg(pkg, torch, local_rank, flush)
    # ---- the paper's example models (throughput; the sweeps run with --paper-only) ----
    pm = paper_models_leg(pkg, torch, local_rank, flush, False)
    vm = vmf_leg(pkg, torch, local_rank)
    # ---- adaptive rank: SVD rule against the learned rank proposer ----
    p2 = None if args.no_ps2 else ps2_leg(args, pkg, torch, local_rank)

    # ---- batched: 256 uneven spin-boson instances in one graph launch per step ----
    batch_out = None
    if not args.no_batch:
        bws = W.spin_boson_batch(n=args.batch)
        hs = [make_gpu(pkg, bw, local_rank) for bw in bws]
        for hh in hs:  # concurrent instances fill the GPU: one CTA per output tile
            hh.ttn_set_params(max_split=1)
        # warps per CTA of the whole batch, by timing (states put back afterwards)
        tune_b = pkg.ttn_batch_autotune(hs, 0.01, 2)
        pkg.ttn_batch_step(hs, 0.01, 1, args.warmup)
        torch.cuda.synchronize()
        s0 = hs[0].stream
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s0):
            flush.zero_()
        ta.record(s0)
        pkg.ttn_batch_step(hs, 0.01, 1, args.steps)
        tb.record(s0)
        torch.cuda.synchronize()
        ms_b = ta.elapsed_time(tb)
        k1 = sum(hh.ttn_stats(0)[1] for hh in hs) / (args.warmup + args.steps)
        rho_b = [hh.ttn_rdm() for hh in hs]
        # the same instances in the mixed form (FP32 contractions, tensor cores
        # for nodes >= 16384 elements), same steps, against the FP64 batch
        hm = [make_gpu(pkg, bw, local_rank, precision=pkg.TTN_MIXED_FP32) for bw in bws]
        for hh in hm:
            hh.ttn_set_params(max_split=1)
        tune_m = pkg.ttn_batch_autotune(hm, 0.01, 2)
        pkg.ttn_batch_step(hm, 0.01, 1, args.warmup)
        torch.cuda.synchronize()
        with torch.cuda.stream(hm[0].stream):
            flush.zero_()
        ta.record(hm[0].stream)
        pkg.ttn_batch_step(hm, 0.01, 1, args.steps)
        tb.record(hm[0].stream)
        torch.cuda.synchronize()
        ms_bm = ta.elapsed_time(tb)
        errs = [float(np.max(np.abs(hh.ttn_rdm() - rb))) for hh, rb in zip(hm, rho_b)]
        scale = [float(np.max(np.abs(rb))) for rb in rho_b]
        bounded = [e for e, sc in zip(errs, scale) if sc <= 1.0 + 1e-9]  # |rho_ij| <= 1 (physical range)
        for hh in hm:
            hh.close()
        # the same instances one after another (each its own step graph), few steps
        n_seq = 2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for hh in hs:
            hh.ttn_step(0.01, 1, n_seq)
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t0
        for hh in hs:
            hh.close()
        batch_out = {"workload": f"{args.batch} spin-boson instances (seeded lambda, omega_c, beta, eps, Delta; "
                                 "K 2-8, depth 6-12, rank 8-32, BTT), ps1 FP64, dt 0.01",
                     "instance_steps_per_s": args.batch * args.steps / (ms_b * 1e-3),
                     "ms_per_batched_step": ms_b / args.steps,
                     "sequential_instance_steps_per_s": args.batch * n_seq / seq_s,
                     "node_contraction_gflop_per_batched_step": k1 / 1e9,
                     "tile_shape": {"how": "ttn_batch_autotune: warps per CTA of every contraction list "
                                           "(8 / 4 / 2) chosen by timing 2 batched steps each; states put back",
                                    "fp64": tune_b, "mixed_fp32": tune_m},
                     "mixed_fp32": {"instance_steps_per_s": args.batch * args.steps / (ms_bm * 1e-3),
                                    "ms_per_batched_step": ms_bm / args.steps,
                                    "rdm_max_abs_vs_fp64_batch": max(errs),
                                    "rdm_max_rel_vs_fp64_batch": max(e / max(1.0, sc) for e, sc in zip(errs, scale)),
                                    "instances_with_max_abs_rho_above_1": len(errs) - len(bounded),
                                    "steps_compared": args.warmup + args.steps},
                     "l2": "one 256 MB flush before the timed batch (the 256 states total ~0.3 GB)"}

    # ---- end to end through the public API with host buffers ----
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2 = make_gpu(pkg, w, local_rank)  # host SOP / rho0 arrays -> device
    rhos = []
    for _ in range(args.steps):
        g2.ttn_step(w.dt, 1, 1)
        rhos.append(g2.ttn_rdm())  # device -> host every step
    e2e_s = time.perf_counter() - t0
    sop = pkg.heom.heom_sop(w.H, w.baths, w.depth, w.drives)
    h2d = sum(np.asarray(v).nbytes for v in sop.values()) + w.rho0.nbytes
    g2.close()
    e2e_s = replica_max(e2e_s, dist, dev)
    peaks = measure_peaks(torch, dev)

    if rank != 0:
        return
    names = {0: "node/bond application (k_apply)", 1: "environment update", 2: "Householder QR", 3: "other"}
    dom = max(range(4), key=lambda k: prof[k][2])
    n_l, fl, t_ms = prof[dom]
    # the class's share of the summed device time of the replayed step graph
    # (event-record nodes) times the step time of the unprofiled timed run:
    # gaps between kernels are attributed in proportion, so this is a lower
    # bound of the kernels' own rate
    prof_sum = sum(p[2] for p in prof.values())
    share = {k: prof[k][2] / prof_sum for k in range(4)} if prof_sum > 0 else {k: 0.0 for k in range(4)}
    t_dom = share[dom] * ms_max
    achieved = (fl / args.steps) / (share[dom] * (ms_max / args.steps) * 1e-3) / 1e12 if share[dom] > 0 else 0.0
    fp64_peak = peaks["fp64_tflops"]
    k1_launches, k1_flops, k1_ms = prof[0]
    value = replicas_value(world, args.steps, ms_max)
    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_nodes": len(w.parent), "state_complex": 83220,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB flush between timed steps (state is L2-resident otherwise)",
                   "launch_shapes": "autotuned (ttn_autotune, %.2f s before the warm-up)" % tune_s
                   if tune_s is not None else "built-in rule"},
        "roofline": {"bound": "alu", "kernel": names[dom], "achieved": achieved,
                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "traffic": APPLY_DRAM_BYTES if names[dom].startswith("node/bond") else None,
                     "traffic_source": "mean dram__bytes_read+write per k_apply launch over the 857 launches of one "
                                       "timed step, ncu (1 pass; caches flushed before each launch) "
                                       "(profiles/apply_traffic_exciton7_r20_fp64.md)",
                     "peak_source": "FP64 torch.matmul 4096^3 measured in this run (peaks.fp64_tflops); "
                                    "nominal FP64 is %.2f" % FP64_PEAK_TFLOPS,
                     "kernel_time": "share of the device time of the replayed step graph (CUDA events recorded "
                                    "as graph nodes, ttn_profile 2) x ms_per_step of the timed run",
                     "kernel_ms_per_step": t_dom / args.steps,
                     "frac_of_nominal_fp64": achieved / FP64_PEAK_TFLOPS,
                     "launches_per_step": n_l / args.steps},
        "node_contraction": {"tflops_kernel": (k1_flops / args.steps) / (share[0] * (ms_max / args.steps) * 1e-3) / 1e12
                             if share[0] > 0 else None,
                             "tflops_step": flops[0] / (ms_max * 1e-3) / 1e12,
                             "gflop_per_step": flops[0] / args.steps / 1e9,
                             "share_of_step_time": share[0]},
        "kernel_time_share": {names[k]: share[k] for k in range(4)},
        "kernel_ms_per_step": {names[k]: share[k] * ms_max / args.steps for k in range(4)},
        "kernel_event_ms_sum_over_step": prof_sum / ms_prof if ms_prof > 0 else None,
        "plain_fp64_steps_per_s": value,
        "mixed_fp32": {"steps_per_s": world * args.steps / (ms_mixed * 1e-3),
                       "speedup_vs_plain_fp64": ms_max / ms_mixed,
                       "rdm_max_abs_vs_fp64_gpu": mixed_err, "steps_compared": n_cmp,
                       "node_contraction_tflops_kernel": (prof_m[0][1] / (prof_m[0][2] * 1e-3) / 1e12)
                       if prof_m[0][2] > 0 else None,
                       "node_contraction_gflop_per_step": mixed_flops / args.steps / 1e9,
                       "kernel_time_share": {names[k]: prof_m[k][2] / sum(p[2] for p in prof_m.values())
                                             for k in range(4)}},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "steps/s",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 16 * w.M * w.M,
                "includes": "handle build, sop_load, workspace bind, rho0 upload, K steps with rho_S read back each step"},
        "batched": batch_out,
        "precision_rank64": r64,
        "config1_spin_boson_tt": c1,
        "ps2_learned_rank": p2,
        "paper_models": pm,
        "vmf": vm,
        "peaks": peaks,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed_region": wall,
    }
    if not args.no_cpu_baseline:
        orc = run_oracle(budget_s=args.cpu_budget, max_steps=args.steps + args.warmup)
        n_o = orc["steps"]
        # GPU trajectory of the same first n_o steps from a fresh state
        g3 = make_gpu(pkg, w, local_rank)
        err = 0.0
        for k in range(n_o):
            g3.ttn_step(w.dt, 1, 1)
            err = max(err, float(np.max(np.abs(g3.ttn_rdm() - orc["rho"][k]))))
        g3.close()
        out["cpu_baseline"] = {"value": n_o / orc["seconds"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                               "sample": f"first {n_o} ps1 steps of the same workload (numpy FP64, 1 thread)",
                               "cpu": cpu_model()}
        ncpu = os.cpu_count() or 1
        orc_all = run_oracle(budget_s=args.cpu_budget, max_steps=args.steps + args.warmup, threads=ncpu)
        out["cpu_baseline_all_cores"] = {
            "value": orc_all["steps"] / orc_all["seconds"], "unit": "steps/s", "cores": ncpu, "kind": "oracle",
            "sample": f"first {orc_all['steps']} ps1 steps (numpy FP64 oracle, BLAS/OpenMP threads = {ncpu}; "
                      "the oracle's per-term products are small, so threads add little)", "cpu": cpu_model()}
        out["rdm_err_vs_oracle"] = {"max_abs": err, "steps_compared": n_o}
    print(json.dumps(out), flush=True)


def bench_reference(args, rank):
    if rank != 0:
        return
    w = workload()
    orc = run_oracle(budget_s=args.cpu_budget * 4, max_steps=args.steps + args.warmup)
    n = orc["steps"]
    v = n / orc["seconds"]
    out = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus, "steps": n,
           "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                            "sample": f"first {n} ps1 steps (numpy FP64 oracle, 1 thread, time-bounded)",
                            "cpu": cpu_model()},
           "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-rank64", action="store_true", help="skip the rank-64 precision leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--no-ps2", action="store_true", help="skip the adaptive-rank / learned-proposer leg")
    ap.add_argument("--tensor-cores", type=int, default=None, choices=[0, 1, 2],
                    help="tensor-core form of the rank-64 mixed leg (library default 1, thread-staged)")
    ap.add_argument("--ps2-only", action="store_true", help="print only the adaptive-rank leg")
    ap.add_argument("--paper-only", action="store_true",
                    help="print only the paper's example models, with the Table 2 convergence sweeps")
    ap.add_argument("--ps2-steps", type=int, default=60)
    ap.add_argument("--ps2-pade", type=int, default=5, help="Pade features of the adaptive-rank workload")
    ap.add_argument("--ps2-cap", type=int, default=32)
    ap.add_argument("--rank64-only", choices=["fp64", "mixed"], default=None,
                    help="profiling aid: run only the rank-64 leg in one form (prints that object, not the bench line)")
    ap.add_argument("--batch", type=int, default=256, help="instances in the batched leg")
    ap.add_argument("--accuracy-steps", type=int, default=0,
                    help="run only a long mixed-vs-FP64 trajectory of this many steps (prints that object)")
    ap.add_argument("--accuracy-every", type=int, default=10, help="compare rho_S every this many steps")
    ap.add_argument("--accuracy-vs", choices=["mixed", "fp64-order"], default="mixed",
                    help="second run of the accuracy trajectory: the mixed form, or FP64 with other launch shapes")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        bench_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        bench_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
