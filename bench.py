"""Benchmark of the shifted randomized ST-HOSVD hot path on GB300.

A step is one pass of the whole path over one synthetic tensor: sketch,
q adaptively shifted power steps, the small SVDs and shift updates, the TTM
shrink of every mode (randomized ST-HOSVD with adaptive shifts) and the
relative-error pass.  Default workload: the 1000 x 1000 x 1000 FP32 tensor
a_ijk = (i^2+j^2+k^2)^(-1/2) plus Gaussian noise at 1e-6 relative, Tucker
rank (50,50,50), oversampling 10, q = 3, in the precision form (power steps
1..q-1 read a bfloat16 copy, the sketch, step q, the TTM and the error read
FP32); the plain FP32 form runs on the same tensor beside it, and a short
serving session (Poisson arrivals) reports p50/p99 latency from arrival.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...      # the FP64 CPU oracle, host cores

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica on its own tensor (the method has no cross-tensor
exchange): weak scaling, max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "shifted-power HBM GB/s (% roofline), tensors/s at stated rel.err; serve p50/p99"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
SMS = 152
MAX_SM_MHZ = 2070.0
# FP32 FFMA issue rate: 128 lanes x 2 flop per SM per clock; FP64 nominal 1.25 TFLOP/s.
FP32_ALU_TFLOPS = SMS * 128 * 2 * MAX_SM_MHZ * 1e6 / 1e12
FP64_TFLOPS = 1.25

WORKLOADS = {
    "tucker400_fp32_st": dict(desc="400^3 FP32 Tucker(20^3, decay 0.8) + 1e-4 noise; "
                                   "randomized ST-HOSVD, adaptive shifts, r=(20,20,20), p=10, q=2",
                              shape=[400, 400, 400], r=[20, 20, 20], s=10, q=2, st=True,
                              dtype="f32", prec=0),
    "tucker400_fp32_st_krgauss": dict(desc="as tucker400_fp32_st with a Khatri-Rao product of "
                                           "Gaussian factors as Omega_k (Section 5.5)",
                                      shape=[400, 400, 400], r=[20, 20, 20], s=10, q=2,
                                      st=True, dtype="f32", prec=0, omega=2),
    "tucker400_fp32_st_holistic": dict(desc="as tucker400_fp32_st with Algorithm B.1: range "
                                            "finder keeps l_k = 30 columns, FP64 ST-HOSVD of "
                                            "the 30^3 tensor, U_k = Q_k V_k",
                                       shape=[400, 400, 400], r=[20, 20, 20], s=10, q=2,
                                       st=True, dtype="f32", prec=0, holistic=True),
    "invradius1000_fp32_st": dict(desc="1000^3 FP32 (i^2+j^2+k^2)^-1/2 + 1e-6 noise; randomized "
                                       "ST-HOSVD, r=(50,50,50), p=10, q=3, plain FP32",
                                  shape=[1000, 1000, 1000], r=[50, 50, 50], s=10, q=3, st=True,
                                  dtype="f32", prec=0, oracle_slices=64),
    "invradius1000_bf16power_st": dict(desc="as invradius1000_fp32_st with power steps 1..q-1 on "
                                            "a bfloat16 copy (precision form)",
                                       shape=[1000, 1000, 1000], r=[50, 50, 50], s=10, q=3,
                                       st=True, dtype="f32", prec=1,
                                       companion="invradius1000_fp32_st", oracle_slices=64),
    "invradius512_bf16power_st": dict(desc="512^3 FP32 (i^2+j^2+k^2)^-1/2 + 1e-6 noise, r=(50,50,50), "
                                           "p=10, q=3, precision form (a small profiling case)",
                                      shape=[512, 512, 512], r=[50, 50, 50], s=10, q=3, st=True,
                                      dtype="f32", prec=1),
    "invradius512_fp32_st": dict(desc="as invradius512_bf16power_st in plain FP32 (a small "
                                      "profiling case)",
                                 shape=[512, 512, 512], r=[50, 50, 50], s=10, q=3, st=True,
                                 dtype="f32", prec=0),
    "superdiag600slow_fp32_st_pve": dict(desc="600^3 FP32 tensor C of Section 5.1 (superdiagonal "
                                              "core v_i = 1/i^2, Haar factors); Algorithm 4: "
                                              "ST-HOSVD with per-mode power counts chosen by "
                                              "the PVE test, tol=0.5, q_max=10, r=(20,20,20), "
                                              "p=10",
                                         shape=[600, 600, 600], r=[20, 20, 20], s=10, q=10,
                                         st=True, dtype="f32", prec=0, pve=0.5),
    "sparse600_fp32_st_pve": dict(desc="600^3 FP32 tensor B of Section 5.1 (600 rank-one terms "
                                       "of 5%-dense vectors, weights 1000/i^2 and 1/i^2); "
                                       "Algorithm 4, tol=0.5, q_max=10, r=(20,20,20), p=10",
                                  shape=[600, 600, 600], r=[20, 20, 20], s=10, q=10, st=True,
                                  dtype="f32", prec=0, pve=0.5),
    "hilbert100_fp64_t": dict(desc="100^3 FP64 Hilbert-type 1/(i+j+k-2); randomized T-HOSVD, "
                                   "r=(10,10,10), p=5, q=1", shape=[100, 100, 100],
                              r=[10, 10, 10], s=5, q=1, st=False, dtype="f64", prec=0),
}
WORKLOADS.update({
    "batch256_fp32_st": dict(desc="256 uneven FP32 instances, order 3 or 4 (1/2 each), sides "
                                  "U[32,160], core ranks U[4,16] (clamped), N(0,1) core, Haar "
                                  "factors, 1e-3 relative noise; randomized ST-HOSVD r = core "
                                  "ranks, p=5, q=2, adaptive shifts, one launch per step kind "
                                  "(work list) inside one CUDA graph; split-K counts from the "
                                  "autotuner", kind="batch", count=256,
                             seed=4, s=5, q=2, dtype="f32", tune=True),
    "serve_poisson200": dict(desc="serving loop: Poisson arrivals at 200 req/s of FP32 3-way "
                                  "tensors, sides from {64,128,256,512,768} per mode, Hilbert-type "
                                  "or Tucker(+1e-3 noise) content 50/50, ranks U[5,40] (< side), "
                                  "q in {1,2,3}, p=10; admission by free pool memory",
                             kind="serve", rate=200.0, duration=60.0, seed=5, s=10,
                             dtype="f32"),
})
DEFAULT_WORKLOAD = "invradius1000_bf16power_st"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# byte of each power-pass kernel class, from one ncu capture of the kernel as
# it stands (summaries under profiles/); a launch's traffic is taken as this
# ratio times its algorithmic bytes (traffic grows in proportion with the
# columns a launch processes).  Absent = not measured for the current code.
#  * power_fused: k_power_tc2 (two W buffers) captured on the 512^3 precision
#    form, mode 1 (268.54 MB read + 3.79 MB written for 268.44 MB of
#    bfloat16 copy).
NCU_TRAFFIC_RATIO = {
    "power_fused": (268.539392e6 + 3.79136e6) / 268.435456e6,
}


# ---- ranks (one process per GPU; replicas, no data-path collective) ----
def rank_seed(base, rank):
    """Each rank's replica draws its own content: seed base + 1000 rank."""
    return base + 1000 * rank


def dist_init(world, local):
    """The process group of a torchrun launch (NCCL), or None for one GPU.
    It carries only barriers and the timing reductions below."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return dist


def max_over_ranks(x, dist, device="cuda"):
    """The whole job's time: the slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist, device="cuda"):
    """Units all ranks processed."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(units_all_ranks, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (ms)."""
    return units_all_ranks / (ms / 1e3)


def make_input(name, rank=0):
    from paper_2506_04840_gb300 import inputs as I
    w = WORKLOADS[name]
    if name.startswith("tucker400"):
        return I.tucker_plus_noise(w["shape"], w["r"], seed=rank_seed(2, rank), noise=1e-4,
                                   decay=0.8, dtype=np.float32)
    if name.startswith("invradius"):
        return I.inverse_radius(w["shape"][0], seed=rank_seed(3, rank), noise=1e-6)
    if name.startswith("sparse600"):
        return I.sparse_rank_one_sum(w["shape"][0], seed=rank_seed(12, rank), dtype=np.float32)
    if name.startswith("superdiag600slow"):
        return I.superdiagonal(w["shape"][0], "slow", seed=rank_seed(11, rank), dtype=np.float32)
    if name.startswith("hilbert100"):
        return I.hilbert(w["shape"])
    raise KeyError(name)


def peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_step(A, w):
    from oracle import tucker as T
    if w.get("pve") is not None:
        G, Us, _, _ = T.rsthosvd_pve(A, w["r"], w["s"], w["q"], w["pve"])
        return T.rel_error(A, G, Us)
    if w.get("holistic"):
        G, Us, _ = T.holistic(A, w["r"], w["s"], w["q"], st=w["st"])
        return T.rel_error(A, G, Us)
    from oracle import omega as om
    kind = om.OMEGA_KINDS[w.get("omega", 0)]
    f = T.rsthosvd if w["st"] else T.rthosvd
    G, Us, _ = f(A, w["r"], w["s"], w["q"], bf16_power=bool(w["prec"]), omega=kind) \
        if w["st"] else f(A, w["r"], w["s"], w["q"], omega=kind)
    return T.rel_error(A, G, Us)


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def config_of(name):
    """The workload's config, printed identically by both arms."""
    w = WORKLOADS[name]
    cfg = {"workload": name, "desc": w["desc"]}
    if w.get("kind") is None:
        nbytes = int(np.prod(w["shape"])) * (8 if w["dtype"] == "f64" else 4)
        cfg["l2"] = ("input (%d MB) larger than L2 (129 MB)" % (nbytes >> 20)
                     if nbytes > 129e6 else "input fits L2")
    elif w["kind"] == "batch":
        from paper_2506_04840_gb300 import inputs as I
        tot = sum(int(np.prod(sh)) * 4 for sh, _, _ in I.batch_specs(w["count"], w["seed"]))
        cfg["l2"] = "inputs (%.1f GB in total) larger than L2 (129 MB)" % (tot / 1e9)
    else:
        cfg["l2"] = "request tensors mostly larger than L2 (129 MB)"
    return cfg


def oracle_sample(name, w, A=None, rank=0):
    """One bounded sample of a single-tensor workload for the oracle:
    (fraction of one tensor it stands for, the sampled tensor, description).
    Workloads with ``oracle_slices`` sample the first that many slices along
    the last mode (same Tucker ranks, same algorithm); cost is counted in
    proportion to the slices, as the streaming passes over modes 1..d-1 are.
    Others take the whole tensor."""
    S = w.get("oracle_slices")
    if S:
        n3 = w["shape"][-1]
        if A is not None:
            As = np.asfortranarray(A[..., :S])
        else:
            from paper_2506_04840_gb300 import inputs as I
            As = I.inverse_radius(w["shape"][0], seed=rank_seed(3, rank), noise=1e-6, slices=S)
        what = ("the first %d of the %d mode-%d slices (%s), counted as %d/%d of a tensor"
                % (S, n3, len(w["shape"]), "x".join(str(x) for x in As.shape), S, n3))
        return S / n3, As, what
    return 1.0, (A if A is not None else make_input(name, rank)), "whole instances of the workload"


def cpu_baseline(name, w, A, budget_s=15.0, max_samples=8):
    """The oracle as it stands on the host cores, on a bounded sample."""
    frac, As, what = oracle_sample(name, w, A)
    n, t0 = 0, time.perf_counter()
    re = None
    while True:
        re = oracle_step(As, w)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= max_samples:
            break
    return {"value": n * frac / el, "unit": "tensors/s", "cores": _cores(), "kind": "oracle",
            "sample": "%s; %d sample(s) in %.1f s (oracle FP64 numpy/LAPACK)" % (what, n, el),
            "rel_err_of_sample": re}


def _oracle_sample_batch(w, budget_s):
    """The oracle on the smallest instances of the batch workload (host copies
    made with the host generator of the same recipe), until budget_s."""
    from oracle import tucker as T
    from paper_2506_04840_gb300 import inputs as I
    specs = sorted(I.batch_specs(w["count"], w["seed"]), key=lambda x: int(np.prod(x[0])))
    n, t0, re = 0, time.perf_counter(), None
    for shape, ranks, sub in specs:
        A = I.tucker_plus_noise(shape, ranks, sub, noise=1e-3, noise_mode="relative",
                                dtype=np.float32).astype(np.float64)
        G, Us, _ = T.rsthosvd(A, ranks, w["s"], w["q"])
        re = T.rel_error(A, G, Us)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return n, el, "the %d smallest of the 256 instances (oracle FP64, %.1f s)" % (n, el), re


def _oracle_sample_serve(w, budget_s):
    from oracle import tucker as T
    from paper_2506_04840_gb300 import inputs as I
    reqs = sorted(I.serving_requests(400, w["seed"], rate=w["rate"]),
                  key=lambda r: int(np.prod(r["shape"])))
    n, t0, re = 0, time.perf_counter(), None
    for rq in reqs:
        A = I.request_tensor(rq).astype(np.float64)
        G, Us, _ = T.rsthosvd(A, rq["ranks"], w["s"], rq["q"])
        re = T.rel_error(A, G, Us)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return n, el, "the %d smallest of 400 requests (oracle FP64, %.1f s)" % (n, el), re


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    if w.get("kind") in ("batch", "serve"):
        fn = _oracle_sample_batch if w["kind"] == "batch" else _oracle_sample_serve
        fn(w, 1.0)                                   # warm-up
        n, el, sample, re = fn(w, 20.0)
        value = n / el
        line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": args.gpus,
                "steps": 1, "warmup": 1, "ms_per_step": 1e3 * el, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference", "config": config_of(args.workload), "rel_err": re,
                "cpu_baseline": {"kind": "oracle", "cores": _cores(), "value": value,
                                 "unit": "tensors/s", "sample": sample},
                "e2e": {"value": value, "unit": "tensors/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    frac, As, what = oracle_sample(args.workload, w)
    for _ in range(args.warmup):
        oracle_step(As, w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        re = oracle_step(As, w)
    el = time.perf_counter() - t0
    value = args.steps * frac / el
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": config_of(args.workload),
            "rel_err": re,
            "cpu_baseline": {"kind": "oracle", "cores": _cores(), "value": value,
                             "unit": "tensors/s", "sample": "each step: " + what},
            "e2e": {"value": value, "unit": "tensors/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _roofline(prof, pk, pk_src, workload):
    """Roofline of the shifted-power pass (the metric's kernel) against the
    measured HBM copy bandwidth: algorithmic bytes per launch (one read of
    the tensor the step works on) over the live CUDA-event launch time.
    The fused tensor-core pass when it ran, else the two CUDA-core halves
    W = X^T Q and Y = X W of each step taken together."""
    kinds = prof["kinds"]
    hbm = float(pk["hbm_gbs"])
    if kinds["power_fused"]["launches"]:
        name = "power_fused"
        kd = kinds[name]
        launches, ms, by = kd["launches"], kd["ms"], kd["bytes"]
        what = "fused shifted-power pass, one read of the bfloat16 copy per step (tcgen05)"
    elif kinds["power_w"]["launches"]:
        name = "power_w+power_y"
        launches = kinds["power_w"]["launches"]
        ms = kinds["power_w"]["ms"] + kinds["power_y"]["ms"]
        by = kinds["power_w"]["bytes"]
        what = ("shifted-power step as two CUDA-core passes (W = X^T Q, Y = X W); "
                "algorithmic bytes = one read of X per step, the kernels read it twice")
    else:
        name = max(kinds, key=lambda k: kinds[k]["ms"])
        kd = kinds[name]
        launches, ms, by = kd["launches"], kd["ms"], kd["bytes"]
        what = "no power step ran (q = 0): the kernel class with the most time"
    launches = max(launches, 1)
    avg_s = ms / launches / 1e3
    per_b = by / launches
    achieved = per_b / avg_s / 1e9 if avg_s > 0 else 0.0
    return name, {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                  "frac": achieved / hbm,
                  "traffic": (NCU_TRAFFIC_RATIO[name] * per_b if name in NCU_TRAFFIC_RATIO
                              else None),
                  "kernel": name, "what": what, "launches": launches,
                  "avg_launch_ms": avg_s * 1e3, "bytes_per_launch": per_b,
                  "peak_source": "HBM copy bandwidth (%s MEASURED_PEAKS.json)" % pk_src
                  if pk_src == "measured" else "fallback 6.8 TB/s"}


def _kernels(prof, steps):
    return {k: {"launches": v["launches"], "ms_per_step": v["ms"] / steps,
                "gbs": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else 0.0,
                "tflops": v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 else 0.0}
            for k, v in prof["kinds"].items() if v["launches"]}


def _latency(prof, steps, ms_per_step):
    """The small svd as a latency line (one CTA per call on a sequential chain)."""
    kd = prof["kinds"]["small_svd"]
    if not kd["launches"]:
        return {}
    return {"small_svd": {"launches_per_step": kd["launches"] / steps,
                          "avg_launch_us": 1e3 * kd["ms"] / kd["launches"],
                          "ms_per_step": kd["ms"] / steps,
                          "share_of_step": (kd["ms"] / steps) / ms_per_step if ms_per_step else None}}


def _power_pass(prof, steps, pk):
    """HBM GB/s of each power-step form that ran: algorithmic bytes (one
    read of the tensor per step) over the summed time of its kernels."""
    kinds = prof["kinds"]
    hbm = float(pk["hbm_gbs"])
    out = {}
    f = kinds["power_fused"]
    if f["launches"]:
        g = f["bytes"] / (f["ms"] / 1e3) / 1e9
        out["bf16_fused"] = {"gbs": g, "frac_of_measured_hbm": g / hbm,
                             "launches_per_step": f["launches"] / steps,
                             "ms_per_step": f["ms"] / steps, "reads_of_x_per_step": 1}
    if kinds["power_w"]["launches"]:
        ms = kinds["power_w"]["ms"] + kinds["power_y"]["ms"] + kinds["ritz"]["ms"]
        g = kinds["power_w"]["bytes"] / (ms / 1e3) / 1e9
        out["fp32_two_pass"] = {"gbs": g, "frac_of_measured_hbm": g / hbm,
                                "steps_per_step": kinds["power_w"]["launches"] / steps,
                                "ms_per_step": ms / steps, "reads_of_x_per_step": 2,
                                "traffic_model_bytes_per_step":
                                    2.0 * kinds["power_w"]["bytes"] / steps,
                                "note": "W = X^T Q and Y = X W each read X (plus the Ritz "
                                        "rotation of the precision form's FP32 step)"}
    return out


def run_batch_workload(args, w, local, world):
    """Many uneven instances as one batch: one launch per step kind over the
    work list, the whole run replayed as one CUDA graph."""
    import torch
    from paper_2506_04840_gb300 import api
    from paper_2506_04840_gb300 import inputs as I
    torch.cuda.set_device(local)
    dist = dist_init(world, local)
    api.load()
    rank = int(os.environ.get("RANK", "0"))
    specs = I.batch_specs(w["count"], rank_seed(w["seed"], rank))
    Ads, cores, Us, rels, items = [], [], [], [], []
    for i, (shape, ranks, sub) in enumerate(specs):
        A = I.tucker_plus_noise_device(shape, ranks, sub, noise=1e-3)
        Ads.append(A)
        cores.append(torch.empty(int(np.prod(ranks)), dtype=torch.float32, device="cuda"))
        Us.append([torch.empty(shape[k] * ranks[k], dtype=torch.float32, device="cuda")
                   for k in range(len(shape))])
        rels.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
        items.append(api.make_item(A, shape, ranks, w["s"], w["q"], cores[-1], Us[-1], rels[-1],
                                   seed=0, tag=i))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    tune = None
    if w.get("tune"):
        # split-K counts from the autotuner (the heuristic is one candidate)
        api.tucker_tune_clear()
        best_ms, heur_ms, shift = api.tucker_tune_batch(items, api.TK_SHIFT_PAPER, stream)
        api.tucker_tune_enable(True)
        tune = {"tuned_ms_per_run": best_ms, "heuristic_ms_per_run": heur_ms,
                "split_scale": 2.0 ** (-shift), "classes": api.tucker_tune_entries(),
                "heuristic_value": w["count"] * 1e3 / heur_ms if heur_ms > 0 else None,
                "note": "tuner's own timing (3 graph runs per candidate); value is the tuned run"}
    h = api.tucker_batch_create(items, api.TK_SHIFT_PAPER, True)
    launches, dev_bytes = api.tucker_batch_info(h)
    for _ in range(args.warmup):
        api.tucker_batch_run(h, stream)
    status, _ = api.tucker_batch_wait(h, len(items))
    assert status == api.TK_OK, status
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        api.tucker_batch_run(h, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    clk = clocks.stop()
    value = job_value(world * w["count"] * args.steps, ms)
    re = np.array([float(r.item()) for r in rels])

    # per-kind breakdown: the same launches without the graph, profiled
    he = api.tucker_batch_create(items, api.TK_SHIFT_PAPER, False)
    api.tucker_profile_enable(True)
    api.tucker_batch_run(he, stream)
    api.tucker_batch_wait(he, len(items))
    prof = api.tucker_profile_read()
    api.tucker_profile_enable(False)
    api.tucker_batch_destroy(he)

    # end to end: inputs from pinned host memory, results back to the host
    try:
        pins = [torch.empty(A.numel(), dtype=torch.float32).pin_memory() for A in Ads]
        pinned = True
    except RuntimeError:
        pins = [torch.empty(A.numel(), dtype=torch.float32) for A in Ads]
        pinned = False
    for pn, A in zip(pins, Ads):
        pn.copy_(A)
    dev_out = cores + [u for U in Us for u in U] + rels
    outs = [torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in dev_out]
    h2d = sum(p.numel() * 4 for p in pins)
    d2h = sum(t.numel() * t.element_size() for t in dev_out)

    # a second set of device inputs and a second batch over them: the
    # host->device copy of step k+1 (copy stream) overlaps the compute of
    # step k; every step's copies and result read-back lie inside the timed
    # region (the outputs are shared: their read-back is ordered on `stream`)
    Ads2 = [torch.empty_like(A) for A in Ads]
    items2 = []
    for i, (shape, ranks, sub) in enumerate(specs):
        items2.append(api.make_item(Ads2[i], shape, ranks, w["s"], w["q"], cores[i], Us[i],
                                    rels[i], seed=0, tag=i))
    h2 = api.tucker_batch_create(items2, api.TK_SHIFT_PAPER, True)
    hb, bufs = [h, h2], [Ads, Ads2]
    cstream = torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    ev_go = torch.cuda.Event()

    def e2e_run(nsteps):
        ev_go.record(stream)
        cstream.wait_event(ev_go)
        with torch.cuda.stream(cstream):
            for pn, A in zip(pins, bufs[0]):
                A.copy_(pn, non_blocking=True)
            ev_in[0].record(cstream)
        for k in range(nsteps):
            b = k & 1
            if k + 1 < nsteps:
                nb = (k + 1) & 1
                with torch.cuda.stream(cstream):
                    if k >= 1:
                        cstream.wait_event(ev_done[nb])
                    for pn, A in zip(pins, bufs[nb]):
                        A.copy_(pn, non_blocking=True)
                    ev_in[nb].record(cstream)
            stream.wait_event(ev_in[b])
            api.tucker_batch_run(hb[b], stream)
            ev_done[b].record(stream)
            for o, t in zip(outs, dev_out):
                o.copy_(t, non_blocking=True)

    e2e_run(2)
    torch.cuda.synchronize()
    ne2e = max(3, args.steps // 2)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_run(ne2e)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist) / ne2e
    api.tucker_batch_destroy(h)
    api.tucker_batch_destroy(h2)
    del Ads2
    pk, pk_src = peaks()
    dom, roof = _roofline(prof, pk, pk_src, args.workload)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (device-generated, seeded)",
            "config": config_of(args.workload),
            "rel_err": float(np.median(re)),
            "batch": {"instances": w["count"], "tensor_gb": sum(A.numel() * 4 for A in Ads) / 1e9,
                      "rel_err_median": float(np.median(re)), "rel_err_max": float(re.max()),
                      "launches_per_step": launches, "device_gb": dev_bytes / 1e9},
            "roofline": roof, "power_pass": _power_pass(prof, 1, pk),
            "latency": _latency(prof, 1, ms / args.steps), "kernels": _kernels(prof, 1),
            "e2e": {"value": world * w["count"] / e2e_s, "unit": "tensors/s",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "host_memory": "pinned" if pinned else "pageable (pinning failed)",
                    "overlap": "step k+1's host->device copy overlaps step k's compute "
                               "(two device input sets, two batches)"},
            "clocks": clk, "gpu_launches": launches * args.steps}
    if tune is not None:
        line["tune"] = tune
        api.tucker_tune_enable(False)
    if world == 1 and not args.no_cpu_baseline:
        n, el, sample, re_o = _oracle_sample_batch(w, 15.0)
        line["cpu_baseline"] = {"value": n / el, "unit": "tensors/s", "cores": _cores(),
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def serve_session(w, duration, rank=0, dist=None, warmup=3, pool=256, server_bytes=0):
    """Poisson arrivals into the serving loop.  The request tensors of a
    pool of ``pool`` requests (the recipe's first ones) are made on the
    device before the arrival clock starts; the arrival stream then replays
    them at the recipe's arrival times, so a submit is only the call itself.
    Latency = completion - scheduled arrival (server clock); the submit lag
    (submit - scheduled arrival) is reported beside it."""
    import torch
    from paper_2506_04840_gb300 import api
    from paper_2506_04840_gb300 import inputs as I
    count = int(w["rate"] * duration)
    reqs = I.serving_requests(count, rank_seed(w["seed"], rank), rate=w["rate"])
    P = min(pool, count)
    hil, content = {}, []
    for rq in reqs[:P]:
        shape = rq["shape"]
        if rq["kind"] == "hilbert":
            key = tuple(shape)
            if key not in hil:
                hil[key] = I.hilbert_device(shape)
            content.append(hil[key])
        else:
            content.append(I.tucker_plus_noise_device(shape, rq["ranks"], rq["seed"], noise=1e-3))

    def spec(i):
        # request i is pool entry i mod P (shape, ranks, q, content)
        return reqs[i % P], content[i % P]

    def outputs(rq):
        core = torch.empty(int(np.prod(rq["ranks"])), dtype=torch.float32, device="cuda")
        U = [torch.empty(rq["shape"][k] * rq["ranks"][k], dtype=torch.float32, device="cuda")
             for k in range(3)]
        rel = torch.zeros(1, dtype=torch.float64, device="cuda")
        return core, U, rel

    # outputs and item descriptors of every request, made before the clock
    items, keep = [], []
    for i in range(count):
        rq, A = spec(i)
        core, U, rel = outputs(rq)
        items.append(api.make_item(A, rq["shape"], rq["ranks"], w["s"], rq["q"], core, U, rel,
                                   seed=0, tag=i % (1 << 24)))
        keep.append((core, U, rel))
    torch.cuda.synchronize()

    srv = api.tucker_server_create(server_bytes, 256, api.TK_SHIFT_PAPER)
    for i in range(min(max(warmup, 3), count)):   # warm-up through the same server
        api.tucker_server_submit(srv, items[i])
    api.tucker_server_drain(srv, 600.0)
    api.tucker_server_poll(srv, 1 << 16)

    api.tucker_profile_enable(True)
    if dist:
        dist.barrier()   # the ranks' arrival streams start together
    t_start = api.tucker_server_clock(srv)
    comps, lag, arrival_of = [], [], {}
    for i, rq in enumerate(reqs):
        while api.tucker_server_clock(srv) - t_start < rq["arrival"]:
            comps.extend(api.tucker_server_poll(srv, 4096))
            time.sleep(0.0001)
        rid = api.tucker_server_submit(srv, items[i])
        arrival_of[rid] = (t_start + rq["arrival"], i)
        lag.append(api.tucker_server_clock(srv) - t_start - rq["arrival"])
    api.tucker_server_drain(srv, 1200.0)
    comps.extend(api.tucker_server_poll(srv, 1 << 16))
    prof = api.tucker_profile_read()
    api.tucker_profile_enable(False)
    api.tucker_server_destroy(srv)
    lat = np.array([c["done_s"] - arrival_of[c["id"]][0] for c in comps]) * 1e3
    span = max(c["done_s"] for c in comps) - t_start
    rels = np.array([float(keep[arrival_of[c["id"]][1]][2].item()) for c in comps])
    bad = sum(1 for c in comps if c["status"] != 0)
    lag_ms = np.array(lag) * 1e3
    return {"completed": len(comps), "failed": bad, "span_s": span, "duration_s": duration,
            "offered_rps": w["rate"], "pool_requests": P,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()),
            "submit_lag_p50_ms": float(np.percentile(lag_ms, 50)),
            "submit_lag_p99_ms": float(np.percentile(lag_ms, 99)),
            "rel_err_median": float(np.median(rels)), "rel_err_max": float(rels.max()),
            "latency_from": "scheduled arrival (server clock)",
            "kernels": prof["kernels"]}


def run_serve_workload(args, w, local, world):
    """The serving workload as the bench's step: requests completed per second."""
    import torch
    from paper_2506_04840_gb300 import api
    torch.cuda.set_device(local)
    dist = dist_init(world, local)
    api.load()
    rank = int(os.environ.get("RANK", "0"))
    duration = args.duration if args.duration else w["duration"]
    clocks = Clocks(local)
    clocks.start()
    sv = serve_session(w, duration, rank, dist, args.warmup)
    clk = clocks.stop()
    # every rank serves its own arrival stream: the job completes the sum of
    # the ranks' requests over the slowest rank's span (latencies: rank 0's)
    value = sum_over_ranks(sv["completed"], dist) / max_over_ranks(sv["span_s"], dist)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": world,
            "steps": sv["completed"], "warmup": max(args.warmup, 3), "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (device-generated pool of requests, seeded)",
            "config": config_of(args.workload), "rel_err": sv["rel_err_median"],
            "serve": sv,
            "e2e": {"value": value, "unit": "tensors/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0,
                    "note": "requests are served from device memory; content is made on the "
                            "device before the arrival clock starts (no host copies)"},
            "clocks": clk, "gpu_launches": sv["kernels"]}
    if world == 1 and not args.no_cpu_baseline:
        n, el, sample, _ = _oracle_sample_serve(w, 15.0)
        line["cpu_baseline"] = {"value": n / el, "unit": "tensors/s", "cores": _cores(),
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--duration", type=float, default=0.0,
                    help="serving workload: seconds of arrivals (default: the workload's)")
    ap.add_argument("--no-serve", action="store_true",
                    help="default workload: skip the short serving session")
    ap.add_argument("--serve-duration", type=float, default=10.0,
                    help="default workload: seconds of arrivals of the serving session")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = WORKLOADS[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    if w.get("kind") == "batch":
        return run_batch_workload(args, w, local, world)
    if w.get("kind") == "serve":
        return run_serve_workload(args, w, local, world)

    import torch
    from paper_2506_04840_gb300 import api
    torch.cuda.set_device(local)
    dist = dist_init(world, local)
    api.load()

    A = make_input(args.workload, rank)
    dims = list(A.shape)
    d = len(dims)
    r = w["r"]
    tdt = torch.float64 if w["dtype"] == "f64" else torch.float32
    ndt = np.float64 if w["dtype"] == "f64" else np.float32
    Ad = api.to_device(A, ndt)
    core = torch.empty(int(np.prod(r)), dtype=tdt, device="cuda")
    U = [torch.empty(dims[k] * r[k], dtype=tdt, device="cuda") for k in range(d)]
    rel = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def make_step(wl):
        """One step of workload wl on the device tensor X (its own workspace)."""
        kind = wl.get("omega", api.TK_OMEGA_GAUSS)
        opts = api.make_opts(d, wl["q"], wl["s"], seed=0, prec=wl["prec"], omega=kind)
        nbytes = (api.tucker_holistic_workspace_size if wl.get("holistic") else
                  api.tucker_workspace_size)(Ad, dims, r, opts, 1 if wl["st"] else 0)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        opts = api.make_opts(d, wl["q"], wl["s"], seed=0, prec=wl["prec"], workspace=ws,
                             omega=kind)
        fn = api.tucker_rsthosvd if wl["st"] else api.tucker_rthosvd
        q_chosen = []

        def step(X):
            if wl.get("pve") is not None:
                qs, _ = api.tucker_rsthosvd_pve(X, dims, r, opts, wl["pve"], core, U,
                                                stream=stream)
                q_chosen[:] = qs
            elif wl.get("holistic"):
                api.tucker_holistic(X, dims, r, opts, 1 if wl["st"] else 0, core, U,
                                    stream=stream)
            else:
                fn(X, dims, r, opts, core, U, stats=False, stream=stream)
            api.tucker_error(X, dims, core, r, U, rel, stream=stream)
        step.ws = ws
        step.q_chosen = q_chosen
        return step

    def timed(step, steps, warmup):
        """CUDA-event time of `steps` device-resident steps, with the
        library's live per-launch events (profile) over the same region."""
        for _ in range(warmup):
            step(Ad)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        api.tucker_profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(Ad)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = api.tucker_profile_read()
        api.tucker_profile_enable(False)
        if dist:
            dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist), prof

    step = make_step(w)
    for _ in range(args.warmup):
        step(Ad)
    torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ms, prof = timed(step, args.steps, 0)
    clk = clocks.stop()
    rel_err = float(rel.item())
    value = job_value(world * args.steps, ms)

    # ---- end to end through the public API, host buffers -----------------
    pin = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=ndt).ravel(order="F"))).pin_memory()
    core_h = torch.empty(core.numel(), dtype=tdt).pin_memory()
    U_h = [torch.empty(u.numel(), dtype=tdt).pin_memory() for u in U]
    rel_h = torch.empty(1, dtype=torch.float64).pin_memory()
    h2d = pin.numel() * pin.element_size()
    d2h = core_h.numel() * core_h.element_size() + sum(u.numel() * u.element_size() for u in U_h) + 8
    # NB device input buffers: the host->device copies (copy stream) run up
    # to NB - 1 steps ahead of the compute, so a copy that is slow now and
    # then (the host side of the link is shared) does not stall the steps;
    # every step's copy and result read-back lie inside the timed region
    NB = 4
    Ae = [torch.empty_like(Ad) for _ in range(NB)]
    cstream = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(NB)]
    ev_done = [torch.cuda.Event() for _ in range(NB)]
    ev_go = torch.cuda.Event()

    def e2e_run(nsteps):
        ev_go.record(stream)
        cstream.wait_event(ev_go)
        issued = 0
        for k in range(nsteps):
            # copies up to step k + NB - 1: copy c reuses the buffer of step
            # c - NB, whose completion event is already enqueued
            while issued < min(nsteps, k + NB):
                c, b = issued, issued % NB
                with torch.cuda.stream(cstream):
                    if c >= NB:
                        cstream.wait_event(ev_done[b])
                    Ae[b].copy_(pin, non_blocking=True)
                    ev_in[b].record(cstream)
                issued += 1
            b = k % NB
            stream.wait_event(ev_in[b])
            step(Ae[b])
            ev_done[b].record(stream)
            core_h.copy_(core, non_blocking=True)
            for uh, ud in zip(U_h, U):
                uh.copy_(ud, non_blocking=True)
            rel_h.copy_(rel, non_blocking=True)

    e2e_run(2)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), dist)
    e2e_value = job_value(world * args.steps, ms_e2e)
    del Ae, pin

    pk, pk_src = peaks()
    dom, roof = _roofline(prof, pk, pk_src, args.workload)
    kernels = _kernels(prof, args.steps)

    # ---- the plain FP32 form on the same tensor (precision-form workloads)
    plain = None
    if w.get("companion"):
        wc = WORKLOADS[w["companion"]]
        step_c = make_step(wc)
        ms_c, prof_c = timed(step_c, args.steps, args.warmup)
        pk2, pk2_src = peaks()
        _, roof_c = _roofline(prof_c, pk2, pk2_src, w["companion"])
        plain = {"workload": w["companion"], "value": job_value(world * args.steps, ms_c),
                 "unit": "tensors/s", "ms_per_step": ms_c / args.steps,
                 "rel_err": float(rel.item()),
                 "speedup_of_precision_form": (ms_c / ms) if ms > 0 else None,
                 "rel_err_ratio_precision_over_plain": rel_err / float(rel.item())
                 if float(rel.item()) > 0 else None,
                 "power_pass": _power_pass(prof_c, args.steps, pk2), "roofline": roof_c,
                 "latency": _latency(prof_c, args.steps, ms_c / args.steps),
                 "kernels": _kernels(prof_c, args.steps)}
        del step_c

    launches = prof["kernels"]
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": w["dtype"], "data": "synthetic", "config": config_of(args.workload),
            "rel_err": rel_err,
            "roofline": roof, "power_pass": _power_pass(prof, args.steps, pk),
            "latency": _latency(prof, args.steps, ms / args.steps), "kernels": kernels,
            "e2e": {"value": e2e_value, "unit": "tensors/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "overlap": "host->device copies run up to three steps ahead of the "
                               "compute (four device input buffers)"},
            "clocks": clk, "gpu_launches": launches}
    if plain is not None:
        line["plain_form"] = plain
    if step.q_chosen:
        line["pve"] = {"tol": w["pve"], "q_max": w["q"], "q_per_mode": list(step.q_chosen)}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, w, A)
    if world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_serve:
        del step, Ad, core, U
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        ws_ = WORKLOADS["serve_poisson200"]
        line["serve"] = dict(workload="serve_poisson200", desc=ws_["desc"],
                             **serve_session(ws_, args.serve_duration, 0, None, 3))
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
