"""Benchmark of the shifted randomized ST-HOSVD hot path on GB300.

A step is one pass of the whole path over one synthetic tensor: sketch,
q adaptively shifted power steps, the small SVDs and shift updates, the TTM
shrink of every mode (randomized ST-HOSVD with adaptive shifts) and the
relative-error pass.  Default workload: a 400 x 400 x 400 FP32 tensor
G x_1 U_1 x_2 U_2 x_3 U_3 + E (G 20^3 N(0,1) scaled by 0.8^(i+j+k), Haar U_k,
E at 1e-4 ||G||/sqrt(N)), Tucker rank (20,20,20), oversampling 10, q = 2.

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
                                  dtype="f32", prec=0),
    "invradius1000_bf16power_st": dict(desc="as invradius1000_fp32_st with power steps 1..q-1 on "
                                            "a bfloat16 copy (precision form)",
                                       shape=[1000, 1000, 1000], r=[50, 50, 50], s=10, q=3,
                                       st=True, dtype="f32", prec=1),
    "invradius512_bf16power_st": dict(desc="512^3 FP32 (i^2+j^2+k^2)^-1/2 + 1e-6 noise, r=(50,50,50), "
                                           "p=10, q=3, precision form (a small profiling case)",
                                      shape=[512, 512, 512], r=[50, 50, 50], s=10, q=3, st=True,
                                      dtype="f32", prec=1),
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
                                  "(work list) inside one CUDA graph", kind="batch", count=256,
                             seed=4, s=5, q=2, dtype="f32"),
    "serve_poisson200": dict(desc="serving loop: Poisson arrivals at 200 req/s of FP32 3-way "
                                  "tensors, sides from {64,128,256,512,768} per mode, Hilbert-type "
                                  "or Tucker(+1e-3 noise) content 50/50, ranks U[5,40] (< side), "
                                  "q in {1,2,3}, p=10; admission by free pool memory",
                             kind="serve", rate=200.0, duration=60.0, seed=5, s=10,
                             dtype="f32"),
})
DEFAULT_WORKLOAD = "tucker400_fp32_st"

# DRAM bytes (read + write) per launch from one ncu capture of the kernel as
# it stands (summaries under profiles/); absent = not measured.
#  * power_fused at 1000^3: k_power_tc2 captured at 512^3 (268.58 MB read,
#    3.80 MB written), reads scaled by the column count (1000^3 / 512^3) and
#    the partial writes by the row count (1000 / 512).
NCU_TRAFFIC = {
    ("invradius512_bf16power_st", "power_fused"): 268.57984e6 + 3.802112e6,
    ("invradius1000_bf16power_st", "power_fused"): 268.57984e6 * (1000 ** 3 / 512 ** 3) +
                                                   3.802112e6 * (1000 / 512),
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


def cpu_baseline(A, w, budget_s=12.0, max_samples=4):
    """The oracle as it stands on the host cores: whole instances of the workload."""
    n, t0 = 0, time.perf_counter()
    re = None
    while True:
        re = oracle_step(A, w)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= max_samples:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": n / el, "unit": "tensors/s", "cores": cores, "kind": "oracle",
            "sample": "%d whole instance(s) of the workload (oracle FP64 numpy/LAPACK, %.1f s)"
                      % (n, el), "rel_err": re}


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


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
                "impl": "reference",
                "config": {"workload": args.workload, "desc": w["desc"], "rel_err": re},
                "cpu_baseline": {"kind": "oracle", "cores": _cores(), "value": value,
                                 "unit": "tensors/s", "sample": sample},
                "e2e": {"value": value, "unit": "tensors/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    A = make_input(args.workload)
    for _ in range(args.warmup):
        oracle_step(A, w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        re = oracle_step(A, w)
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    value = args.steps / el
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": w["desc"], "rel_err": re},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value,
                             "unit": "tensors/s",
                             "sample": "each step one whole instance of the workload"},
            "e2e": {"value": value, "unit": "tensors/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _roofline(prof, pk, pk_src, fp64=False):
    kinds = prof["kinds"]
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    kd = kinds[dom]
    avg_s = kd["ms"] / max(kd["launches"], 1) / 1e3
    per_b = kd["bytes"] / max(kd["launches"], 1)
    per_f = kd["flops"] / max(kd["launches"], 1)
    if dom == "power_fused":
        bound, unit, achieved = "hbm", "GB/s", per_b / avg_s / 1e9
        peak, note = float(pk["hbm_gbs"]), "HBM copy bandwidth (%s)" % pk_src
    elif fp64:
        bound, unit, achieved = "alu", "TFLOP/s", per_f / avg_s / 1e12
        peak, note = FP64_TFLOPS, "FP64 nominal 1.25 TFLOP/s (recipe table)"
    else:
        bound, unit, achieved = "alu", "TFLOP/s", per_f / avg_s / 1e12
        peak, note = FP32_ALU_TFLOPS, "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz"
    return dom, {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                 "frac": achieved / peak, "kernel": dom, "launches": kd["launches"],
                 "avg_launch_ms": avg_s * 1e3, "bytes_per_launch": per_b,
                 "flops_per_launch": per_f, "peak_source": note}


def _kernels(prof, steps):
    return {k: {"launches": v["launches"], "ms_per_step": v["ms"] / steps,
                "gbs": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else 0.0,
                "tflops": v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 else 0.0}
            for k, v in prof["kinds"].items() if v["launches"]}


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
    dom, roof = _roofline(prof, pk, pk_src)
    roof["traffic"] = NCU_TRAFFIC.get((args.workload, dom))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (device-generated, seeded)",
            "config": {"workload": args.workload, "desc": w["desc"], "instances": w["count"],
                       "tensor_gb": sum(A.numel() * 4 for A in Ads) / 1e9,
                       "rel_err_median": float(np.median(re)), "rel_err_max": float(re.max()),
                       "launches_per_step": launches, "device_gb": dev_bytes / 1e9,
                       "l2": "inputs (%.1f GB) larger than L2 (129 MB)"
                             % (sum(A.numel() * 4 for A in Ads) / 1e9)},
            "roofline": roof, "kernels": _kernels(prof, 1),
            "e2e": {"value": world * w["count"] / e2e_s, "unit": "tensors/s",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "host_memory": "pinned" if pinned else "pageable (pinning failed)",
                    "overlap": "step k+1's host->device copy overlaps step k's compute "
                               "(two device input sets, two batches)"},
            "clocks": clk, "gpu_launches": launches * args.steps}
    if world == 1 and not args.no_cpu_baseline:
        n, el, sample, re_o = _oracle_sample_batch(w, 15.0)
        line["cpu_baseline"] = {"value": n / el, "unit": "tensors/s", "cores": _cores(),
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_serve_workload(args, w, local, world):
    """Poisson arrivals into the serving loop; latency = completion - submit."""
    import torch
    from paper_2506_04840_gb300 import api
    from paper_2506_04840_gb300 import inputs as I
    torch.cuda.set_device(local)
    dist = dist_init(world, local)
    api.load()
    rank = int(os.environ.get("RANK", "0"))
    duration = args.duration if args.duration else w["duration"]
    count = int(w["rate"] * duration)
    reqs = I.serving_requests(count, rank_seed(w["seed"], rank), rate=w["rate"])
    hil = {}
    # warm-up: a few requests through a scratch server
    srv = api.tucker_server_create(0, 256, api.TK_SHIFT_PAPER)
    live = {}

    def make(rq, tag):
        shape = rq["shape"]
        if rq["kind"] == "hilbert":
            key = tuple(shape)
            if key not in hil:
                hil[key] = I.hilbert_device(shape)
            A = hil[key]
        else:
            A = I.tucker_plus_noise_device(shape, rq["ranks"], rq["seed"], noise=1e-3)
        core = torch.empty(int(np.prod(rq["ranks"])), dtype=torch.float32, device="cuda")
        U = [torch.empty(shape[k] * rq["ranks"][k], dtype=torch.float32, device="cuda")
             for k in range(3)]
        rel = torch.zeros(1, dtype=torch.float64, device="cuda")
        it = api.make_item(A, shape, rq["ranks"], w["s"], rq["q"], core, U, rel, seed=0,
                           tag=tag % (1 << 24))
        return it, (A, core, U, rel)

    for i, rq in enumerate(reqs[:max(args.warmup, 3)]):
        it, keep = make(rq, i)
        torch.cuda.current_stream().synchronize()
        live[api.tucker_server_submit(srv, it)] = keep
    api.tucker_server_drain(srv, 600.0)
    api.tucker_server_poll(srv, 1 << 16)
    live.clear()

    api.tucker_profile_enable(True)
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()   # the ranks' arrival streams start together
    t_start = api.tucker_server_clock(srv)
    comps, lag, rels = [], [], {}
    for i, rq in enumerate(reqs):
        while api.tucker_server_clock(srv) - t_start < rq["arrival"]:
            for c in api.tucker_server_poll(srv, 4096):
                comps.append(c)
                rels[c["id"]] = live.pop(c["id"])[3]
            time.sleep(0.0002)
        it, keep = make(rq, i)
        torch.cuda.current_stream().synchronize()   # content ready before the server reads it
        rid = api.tucker_server_submit(srv, it)
        live[rid] = keep
        lag.append(api.tucker_server_clock(srv) - t_start - rq["arrival"])
    api.tucker_server_drain(srv, 1200.0)
    for c in api.tucker_server_poll(srv, 1 << 16):
        comps.append(c)
        rels[c["id"]] = live.pop(c["id"])[3]
    clk = clocks.stop()
    prof = api.tucker_profile_read()
    api.tucker_profile_enable(False)
    api.tucker_server_destroy(srv)
    lat = np.array([c["done_s"] - c["submit_s"] for c in comps]) * 1e3
    span = max(c["done_s"] for c in comps) - min(c["submit_s"] for c in comps)
    # every rank serves its own arrival stream: the job completes the sum of
    # the ranks' requests over the slowest rank's span (latencies: rank 0's)
    value = sum_over_ranks(len(comps), dist) / max_over_ranks(span, dist)
    re = np.array([float(r.item()) for r in rels.values()])
    bad = sum(1 for c in comps if c["status"] != 0)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": world,
            "steps": len(comps), "warmup": max(args.warmup, 3), "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (device-generated per request, seeded)",
            "config": {"workload": args.workload, "desc": w["desc"], "duration_s": duration,
                       "offered_rps": w["rate"], "requests": len(comps), "failed": bad,
                       "rel_err_median": float(np.median(re)), "rel_err_max": float(re.max()),
                       "l2": "request tensors mostly larger than L2"},
            "serve": {"p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)),
                      "mean_ms": float(lat.mean()),
                      "submit_lag_p99_ms": float(np.percentile(np.array(lag) * 1e3, 99))},
            "e2e": {"value": value, "unit": "tensors/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0,
                    "note": "requests are served from device memory; content is made on the "
                            "device per request (no host copies)"},
            "clocks": clk, "gpu_launches": prof["kernels"]}
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
    kind = w.get("omega", api.TK_OMEGA_GAUSS)
    opts = api.make_opts(d, w["q"], w["s"], seed=0, prec=w["prec"], omega=kind)
    nbytes = (api.tucker_holistic_workspace_size if w.get("holistic") else
              api.tucker_workspace_size)(Ad, dims, r, opts, 1 if w["st"] else 0)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    opts = api.make_opts(d, w["q"], w["s"], seed=0, prec=w["prec"], workspace=ws, omega=kind)
    fn = api.tucker_rsthosvd if w["st"] else api.tucker_rthosvd
    stream = torch.cuda.current_stream()

    q_chosen = []

    def step(X):
        if w.get("pve") is not None:
            qs, _ = api.tucker_rsthosvd_pve(X, dims, r, opts, w["pve"], core, U, stream=stream)
            q_chosen[:] = qs
        elif w.get("holistic"):
            api.tucker_holistic(X, dims, r, opts, 1 if w["st"] else 0, core, U, stream=stream)
        else:
            fn(X, dims, r, opts, core, U, stats=False, stream=stream)
        api.tucker_error(X, dims, core, r, U, rel, stream=stream)

    for _ in range(args.warmup):
        step(Ad)
    torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    api.tucker_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(Ad)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = api.tucker_profile_read()
    api.tucker_profile_enable(False)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist)
    rel_err = float(rel.item())
    value = job_value(world * args.steps, ms)

    # ---- end to end through the public API, host buffers -----------------
    pin = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=ndt).ravel(order="F"))).pin_memory()
    core_h = torch.empty(core.numel(), dtype=tdt).pin_memory()
    U_h = [torch.empty(u.numel(), dtype=tdt).pin_memory() for u in U]
    rel_h = torch.empty(1, dtype=torch.float64).pin_memory()
    h2d = pin.numel() * pin.element_size()
    d2h = core_h.numel() * core_h.element_size() + sum(u.numel() * u.element_size() for u in U_h) + 8
    # two device input buffers: the host->device copy of step k+1 (copy
    # stream) overlaps the compute of step k; every step's copy and result
    # read-back lie inside the timed region
    Ae = [torch.empty_like(Ad), torch.empty_like(Ad)]
    cstream = torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    ev_go = torch.cuda.Event()

    def e2e_run(nsteps):
        ev_go.record(stream)
        cstream.wait_event(ev_go)
        with torch.cuda.stream(cstream):
            Ae[0].copy_(pin, non_blocking=True)
            ev_in[0].record(cstream)
        for k in range(nsteps):
            b = k & 1
            if k + 1 < nsteps:
                nb = (k + 1) & 1
                with torch.cuda.stream(cstream):
                    if k >= 1:
                        cstream.wait_event(ev_done[nb])   # step k-1 read buffer nb
                    Ae[nb].copy_(pin, non_blocking=True)
                    ev_in[nb].record(cstream)
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
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), dist)
    e2e_value = job_value(world * args.steps, ms_e2e)

    # ---- roofline of the dominant kernel ----------------------------------
    pk, pk_src = peaks()
    kinds = prof["kinds"]
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    kd = kinds[dom]
    avg_s = kd["ms"] / max(kd["launches"], 1) / 1e3
    per_launch_bytes = kd["bytes"] / max(kd["launches"], 1)
    per_launch_flops = kd["flops"] / max(kd["launches"], 1)
    if dom == "power_fused":
        bound, unit = "hbm", "GB/s"
        achieved = per_launch_bytes / avg_s / 1e9
        peak = float(pk["hbm_gbs"])
        peak_note = "HBM copy bandwidth (%s)" % pk_src
    elif w["dtype"] == "f64":
        bound, unit = "alu", "TFLOP/s"
        achieved = per_launch_flops / avg_s / 1e12
        peak = FP64_TFLOPS
        peak_note = "FP64 nominal 1.25 TFLOP/s (recipe table)"
    else:
        bound, unit = "alu", "TFLOP/s"
        achieved = per_launch_flops / avg_s / 1e12
        peak = FP32_ALU_TFLOPS
        peak_note = "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": NCU_TRAFFIC.get((args.workload, dom)),
            "kernel": dom, "launches": kd["launches"], "avg_launch_ms": avg_s * 1e3,
            "bytes_per_launch": per_launch_bytes, "flops_per_launch": per_launch_flops,
            "peak_source": peak_note}
    hbm_frac = {k: (v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else 0.0)
                for k, v in kinds.items()}
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                   "gbs": round(hbm_frac[k], 1),
                   "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 else 0.0)}
               for k, v in kinds.items() if v["launches"]}

    # the shifted-power pass (fused, or the two CUDA-core halves) as HBM GB/s
    pw = [kinds[k] for k in ("power_fused", "power_w", "power_y") if kinds[k]["launches"]]
    pw_ms = sum(v["ms"] for v in pw)
    pw_gbs = ((kinds["power_fused"]["bytes"] + kinds["power_w"]["bytes"]) / (pw_ms / 1e3) / 1e9
              if pw_ms > 0 else 0.0)
    power_pass = {"gbs": pw_gbs, "frac_of_measured_hbm": pw_gbs / float(pk["hbm_gbs"]),
                  "fused_traffic_per_launch": NCU_TRAFFIC.get((args.workload, "power_fused")),
                  "ms_per_step": pw_ms / args.steps,
                  "note": "algorithmic bytes of X read once per power step / summed time of "
                          "the power kernels"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": "tensors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": w["dtype"], "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "rel_err": rel_err,
                       "l2": "input (%d MB) larger than L2 (129 MB)" % (Ad.numel() *
                                                                       Ad.element_size() >> 20)
                       if Ad.numel() * Ad.element_size() > 129e6 else "input fits L2"},
            "roofline": roof, "power_pass": power_pass, "kernels": kernels,
            "e2e": {"value": e2e_value, "unit": "tensors/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "overlap": "step k+1's host->device copy overlaps step k's compute "
                               "(two device input buffers)"},
            "clocks": clk, "gpu_launches": prof["kernels"]}
    if q_chosen:
        line["config"]["pve"] = {"tol": w["pve"], "q_max": w["q"], "q_per_mode": list(q_chosen)}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, w)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
