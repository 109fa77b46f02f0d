"""Benchmark: exact three-hop top-K path search, queries/s on GB300.

Default workload (N = 1): the batching configuration, R-MAT typed knowledge
graph with 10,000,000 vertices, 200,000,000 edges, 32 relations, 6 vertex
types, d = 128 bf16 embeddings ~ N(0, 1/sqrt(d)); 4,096 (s, t) queries with
log-uniform source degree in [1, 1e5], K = 50, TransE-L1 score (--workload
medium: 1,000,000 vertices / 20,000,000 edges, d = 128 fp32, 64 queries,
K = 100).  A step is one batched call that runs the whole path for all the
workload's queries (hop-1 / hop-3 expansion, direction choice, middle join,
streaming top-K, fp64 rescoring, final order).  With torchrun (N > 1) every
rank runs its own queries on a replica of the graph (weak scaling, no
data-path collective).

Output: one JSON line on rank 0.
  value       queries/s over all ranks, device-timed (CUDA events around each
              step on the launch stream; L2 flushed before every step; inputs
              resident in HBM)
  e2e         the same metric through the C ABI with host buffers: host->device
              copy of the queries and device->host copy of the results inside
              the timed region (wall clock)
  roofline    middle-join kernel: algorithmic bytes / its event-timed duration
              against the measured HBM copy bandwidth
  cpu_baseline the CPU oracle (fp64 brute force, OpenMP over queries) on a
              bounded sample of the same queries
  oracle_parity every query of that sample compared with the GPU result
  precision_error fp32 screening error of every returned path against its
              fp64 score, next to the proven bound

--workload tail measures the tail-prediction scan (Alg. 3 / Alg. 4) and
--workload beam the H-hop beam search (Alg. 6 / Alg. 7), each with its own
JSON line; the other workloads are extra measurements of the three-hop search.

--impl reference runs the CPU oracle as the reference arm on the same
workload (bounded samples per step) and prints the same JSON line.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3-hop top-K queries/s on 1 GB300, plain vs chosen form, top-K identical to oracle"
UNIT = "queries/s"
WORKLOAD = "batching"
WORKLOAD_DESCS = {
    "medium": ("R-MAT (a,b,c)=(.57,.19,.19) typed KG: 1,000,000 vertices, 20,000,000 edges, "
               "16 relations, 6 vertex types, d=128 fp32 embeddings ~N(0,1/sqrt(d)); "
               "64 edge-biased (s,t) queries per step, K=100, TransE-L1 (gamma=1)"),
    "batching": ("R-MAT (a,b,c)=(.57,.19,.19) typed KG: 10,000,000 vertices, 200,000,000 edges, "
                 "32 relations, 6 vertex types, d=128 bf16 embeddings ~N(0,1/sqrt(d)); 4,096 queries "
                 "per step with log-uniform source degree in [1,1e5], K=50, TransE-L1 (gamma=1)"),
    "batching_quarter": ("the batching recipe at a quarter of its size (the profiler-capture case): R-MAT "
                         "(a,b,c)=(.57,.19,.19) typed KG: 2,500,000 vertices, 50,000,000 edges, 32 relations, "
                         "6 vertex types, d=128 bf16 embeddings ~N(0,1/sqrt(d)); 1,024 queries per step with "
                         "log-uniform source degree in [1,1e5], K=50, TransE-L1 (gamma=1)"),
    "tiny": ("Zipf(2.1) typed KG: 10,000 vertices, 100,000 edges, 8 relations, d=64 fp32 ~N(0,1/8); "
             "one hub query, K=10, TransE-L1"),
    "precision": ("the medium R-MAT graph (1,000,000 vertices, 20,000,000 edges, 16 relations) with d=256 "
                  "fp32 embeddings ~N(0,1/sqrt(d)); 256 edge-biased queries per step, K=100, DistMult"),
    "learned": ("the precision workload's graph and 256 queries (d=256 fp32, DistMult) with K=50 "
                "(or the K given), ordering MLP trained on 20,000 held-out queries"),
    "beam": ("generic H-hop search with a per-path beam (Alg. 6 / Alg. 7) on the medium graph "
             "(1,000,000 vertices, d=128 fp32, TransE-L1): the medium workload's 64 (s,t) queries, H=3, "
             "beam K=10, the 10 best paths per query"),
    "tail": ("tail prediction (Alg. 3 / Alg. 4) on the medium graph (1,000,000 vertices, d=128 fp32, "
             "TransE-L1): a step scores 64 heads (the K persons of Alg. 4), each with its own relation, "
             "against every vertex of type 0 (~166,700 candidates), K=50; single-head line: one head "
             "against all 1,000,000 vertices (Alg. 3), K=50"),
}
K_OVERRIDE = 0
WORKLOAD_DESC = WORKLOAD_DESCS[WORKLOAD]
DATA = "synthetic: seeded R-MAT typed knowledge graph standing in for WikiKG90Mv2"
FORM_DESC = {"plain": "plain: batched, every middle edge scored, fp32 screen + fp64 rescoring",
             "bound": "bound: plain + rows ordered by their score bound, a seed pass per query, provable "
                      "bound pruning of work items, rows and hits (identical output)",
             "chosen": "chosen: as bound, with rows ordered by the learned MLP score (trained on plain runs "
                       "over 20,000 held-out queries before timing) (identical output)"}
# kernels per step: k_init, k_expand_v, scan x2, k_lists, k_plan, k_order_key, k_mlp_qbias,
# k_mlp_keys, k_order_hist, scan x2, k_order_perm, scan x2, k_near, k_middle (seed),
# k_middle, k_merge1, k_rescore, k_merge2, k_exact
KERNELS_PER_STEP = 22
# DRAM bytes (read + write) of one main join launch from one ncu capture of the
# current kernel, per (workload, form, work-item size, scan tile); any other
# configuration reports null.
TRAFFIC_NCU = {# batching workload: the main join launch of the first timed step, one
               # capture of the current kernel (1 pass: dram__bytes_read.sum +
               # dram__bytes_write.sum at full size, --profile-range)
               ("batching", "chosen", 32768, 4): 143_070_000_000}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_queries(g, S, T, rank: int, workload: str):
    """Weak scaling: rank 0 keeps the workload's queries, rank r > 0 draws its own
    set of the same size and recipe (seed r) on the same graph."""
    import synth
    if rank == 0:
        return S, T
    if synth.WORKLOADS[workload]["queries"] == "logdeg":
        return synth.queries_log_degree(g, len(S), seed=rank)
    return synth.queries_edge_biased(g, len(S), seed=rank)


def max_over_ranks(x: float, ws: int, device) -> float:
    """The job's time is the slowest rank's: all-reduce MAX (no-op at N = 1)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def init_replicas(ws: int, local: int):
    """One process per GPU under torchrun: the process group carries only the
    timing reduction (replicas, no data-path collective)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))


def close_replicas(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def job_rate(units_per_rank: int, ws: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return units_per_rank * ws * steps / (max_ms / 1000.0)


def load_workload(rank: int):
    import synth
    os.environ.setdefault("MHR_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "mhr_synth_cache"))
    g, S, T, K, spec = synth.workload(WORKLOAD)
    S, T = rank_queries(g, S, T, rank, WORKLOAD)
    if K_OVERRIDE:
        K = K_OVERRIDE
    return g, S, T, K, spec


# ------------------------------------------------------------------ graph statistics
def frontier_stats(g, S, T):
    """|U|, |V_t|, S_f, S_b per query from the graph arrays (numpy)."""
    od = np.diff(g.offsets)
    order = np.argsort(g.cols, kind="stable")
    src = g.src_of_edges()[order]
    indeg = np.bincount(g.cols, minlength=g.n).astype(np.int64)
    roff = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(indeg, out=roff[1:])
    out = []
    for s, t in zip(S.tolist(), T.tolist()):
        U = np.unique(g.cols[g.offsets[s]:g.offsets[s + 1]])
        U = U[(U != s) & (U != t)]
        V = np.unique(src[roff[t]:roff[t + 1]])
        V = V[(V != s) & (V != t)]
        out.append(dict(deg_s=int(od[s]), deg_t=int(indeg[t]), n_u=int(U.size), n_v=int(V.size),
                        s_f=int(od[U].sum()), s_b=int(indeg[V].sum())))
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="mhr_clocks_", suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle legs
def cpu_oracle_rate(g, S, T, K, budget_s: float = 30.0, fn: str = "transe"):
    """The oracle (unchanged) on a bounded prefix sample of the queries.
    Returns (cpu_baseline dict, (n, paths, n_paths) of the last sample run)."""
    import oracle
    oracle.build()
    n = 1
    best = None
    while True:
        t0 = time.perf_counter()
        want, n_want = oracle.topk_paths_batch(g, S[:n], T[:n], K, fn=fn)
        dt = time.perf_counter() - t0
        best = (n, dt, want, n_want)
        if n >= len(S) or dt > budget_s / 3:
            break
        n = min(len(S), n * 2)
    n, dt, want, n_want = best
    return ({"value": n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
             "sample": f"first {n} of the {len(S)} workload queries, fp64 brute force, "
                       f"OpenMP over queries, {dt:.2f} s"}, (n, want, n_want))


def oracle_parity(dev_paths, dev_n, sample):
    """Every query the CPU oracle computed, compared with the GPU result of the
    timed form: count and order of paths, (u, r1, v, r2, r3) of each path and
    its fp64 score, all bit-exact."""
    n, want, n_want = sample
    bad = []
    for q in range(n):
        k = int(n_want[q])
        if int(dev_n[q]) != k:
            bad.append(q)
            continue
        a, b = dev_paths[q][:k], want[q][:k]
        if not all(np.array_equal(a[f], b[f]) for f in ("u", "r1", "v", "r2", "r3")):
            bad.append(q)
            continue
        if a["score"].tobytes() != b["score"].tobytes():
            bad.append(q)
    return {"checked": n, "mismatches": len(bad), "first_mismatch": (bad[0] if bad else None),
            "paths_compared": int(sum(int(n_want[q]) for q in range(n))),
            "rule": "the first n workload queries (the CPU baseline's sample): path count, ids, order and "
                    "fp64 scores bit-exact against the oracle"}


def precision_error(mhr, G, S, T, paths, n_out):
    """Error of the fp32 screening arithmetic against fp64, over every path the
    step returned: S32 = fl32(fl32(w1 + w2) + w3) from the library's fp32 edge
    weights, S64 = the returned (fp64, exact) score; with the proven bound E
    on |S32 - S64| the screen keeps every path within 2E of the K-th score."""
    info = mhr.mhr_graph_get_info(G)
    src, rel, dst, s64 = [], [], [], []
    for q in range(len(S)):
        k = int(n_out[q])
        if k <= 0:
            continue
        p = paths[q][:k]
        s, t = np.uint32(S[q]), np.uint32(T[q])
        src += [np.full(k, s, np.uint32), p["u"], p["v"]]
        rel += [p["r1"], p["r2"], p["r3"]]
        dst += [p["u"], p["v"], np.full(k, t, np.uint32)]
        s64.append(p["score"])
    if not s64:
        return None
    m = sum(x.size for x in s64)
    # edges grouped per query as [hop1 | hop2 | hop3] blocks of k
    src, rel, dst = np.concatenate(src), np.concatenate(rel).astype(np.uint16), np.concatenate(dst)
    w = mhr.mhr_edge_scores(G, src, rel, dst, precision=0)
    w1, w2, w3, pos = [], [], [], 0
    for x in s64:
        k = x.size
        w1.append(w[pos:pos + k])
        w2.append(w[pos + k:pos + 2 * k])
        w3.append(w[pos + 2 * k:pos + 3 * k])
        pos += 3 * k
    w1, w2, w3 = np.concatenate(w1), np.concatenate(w2), np.concatenate(w3)
    s32 = ((w1 + w2).astype(np.float32) + w3).astype(np.float32).astype(np.float64)
    s64 = np.concatenate(s64)
    ae = np.abs(s32 - s64)
    re = ae / np.maximum(np.abs(s64), 1e-300)
    E = info["err_path"]
    return {"paths": int(m), "max_abs": float(ae.max()), "mean_abs": float(ae.mean()),
            "max_rel": float(re.max()), "mean_rel": float(re.mean()), "bound_E": E,
            "max_abs_over_E": float(ae.max() / E), "eps32_edge": info["eps32_edge"],
            "what": "S32 = fp32 sum of the library's fp32 edge weights vs the returned fp64 score, every "
                    "returned path of one step; E = proven bound on |S32 - S64| per path"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    metric = METRIC
    if WORKLOAD == "tail":
        import synth
        os.environ.setdefault("MHR_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "mhr_synth_cache"))
        g = synth.workload("medium")[0]
        S, T = tail_queries(g, TAIL_NQ, 0)
        metric = TAIL_METRIC
    elif WORKLOAD == "beam":
        import synth
        os.environ.setdefault("MHR_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "mhr_synth_cache"))
        g, S, T, _, _ = synth.workload("medium")
        metric = BEAM_METRIC
    else:
        g, S, T, K, spec = load_workload(0)
    fn = spec.get("score", "transe") if WORKLOAD not in ("tail", "beam") else "transe"
    # Every step runs the same batch of queries through the oracle (OpenMP over
    # the batch, dynamic schedule): queries spaced evenly through the workload's
    # list, so the sample spans its degree mix.  The batch is sized once, by
    # doubling from one query per thread until a batch takes the per-step
    # budget, so the whole run stays within a few minutes.
    cores = oracle.num_threads()
    budget = min(6.0, max(0.3, 150.0 / (args.warmup + args.steps)))

    def sample(m):
        return np.unique(np.linspace(0, len(S) - 1, m).round().astype(np.int64))

    def run(idx):
        t0 = time.perf_counter()
        if WORKLOAD == "tail":
            oracle.tail_topk(g, S[idx], T[idx], TAIL_K, cand_type=TAIL_TYPE)
        elif WORKLOAD == "beam":
            oracle.beam_paths_batch(g, S[idx], T[idx], BEAM_H, BEAM_K)
        else:
            oracle.topk_paths_batch(g, S[idx], T[idx], K, fn=fn)
        return time.perf_counter() - t0

    per_step = max(1, min(len(S), cores))
    while per_step < len(S) and run(sample(per_step)) < budget:
        per_step = min(len(S), 2 * per_step)
    idx = sample(per_step)
    per_step = len(idx)
    times = []
    for step in range(args.warmup + args.steps):
        dt = run(idx)
        if step >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step * len(times) / tot
    line = {"impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA,
            "config": {"workload": WORKLOAD_DESC, "queries_per_step": per_step,
                       "note": (f"CPU oracle: fp64 beam search, OpenMP over the step's {per_step} queries"
                                if WORKLOAD == "beam" else
                                f"CPU oracle: fp64 brute force, OpenMP over the step's {per_step} queries")},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} queries per step (one batch, sized to about {budget:.1f} s), "
                                       f"spaced evenly through the {len(S)} workload queries, the same "
                                       f"batch every step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ tail prediction
TAIL_NQ, TAIL_K, TAIL_TYPE = 64, 50, 0
TAIL_METRIC = "tail-prediction queries/s (Alg. 3 / Alg. 4) on 1 GB300, top-K identical to oracle"
TAIL_KERNELS_PER_CALL = 4   # sampling scan, sampling threshold, full scan, final select + rescoring


def tail_queries(g, nq, seed):
    rng = np.random.default_rng(1000 + seed)
    return (rng.integers(0, g.n, size=nq).astype(np.uint32),
            rng.integers(0, g.R, size=nq).astype(np.uint16))


def run_tail(args):
    """Tail-prediction scan: device-timed calls with inputs resident in HBM,
    L2 flushed before every call; roofline of the full-scan kernel."""
    import torch
    import synth
    import paper_2406_07727_gb300 as mhr

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_replicas(ws, local)
    os.environ.setdefault("MHR_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "mhr_synth_cache"))
    g = synth.workload("medium")[0]
    G = mhr.load_kg(g)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    H, Rq = tail_queries(g, TAIL_NQ, rank)
    dH = torch.from_numpy(H.astype(np.int32)).cuda()
    dR = torch.from_numpy(Rq.astype(np.int16)).cuda()
    n_cand = int(np.sum(g.vtypes == TAIL_TYPE))
    eb = 4 if g.dtype == "f32" else 2

    def measure(hq, rq, nq, cand_type, steps):
        out = torch.empty((nq, TAIL_K * 16), dtype=torch.uint8, device="cuda")
        n_out = torch.empty(nq, dtype=torch.int32, device="cuda")
        for _ in range(args.warmup):
            mhr.mhr_tail_topk(G, hq, rq, TAIL_K, cand_type=cand_type, out=out, n_out=n_out, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        scan_ms, stats = [], None
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            _, _, stats = mhr.mhr_tail_topk(G, hq, rq, TAIL_K, cand_type=cand_type, out=out, n_out=n_out,
                                            stream=stream, with_stats=True)
            ev[i][1].record(stream)
            scan_ms.append(stats["ms_join"])
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return sum(ms), statistics.mean(scan_ms), stats, out, n_out

    clocks = ClockSampler(local)
    clocks.start()
    tot_ms, scan_ms, st, out, n_out = measure(dH, dR, TAIL_NQ, TAIL_TYPE, args.steps)
    clk = clocks.stop()
    value = job_rate(TAIL_NQ, ws, args.steps, max_over_ranks(tot_ms, ws, "cuda"))
    # single head against every vertex (Alg. 3)
    s_steps = max(3, args.steps // 4)
    tot1, scan1, st1, _, _ = measure(dH[:1], dR[:1], 1, -1, s_steps)

    # end to end with host buffers
    e2e = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h_out, h_n = mhr.mhr_tail_topk(G, H, Rq, TAIL_K, cand_type=TAIL_TYPE)
        e2e.append(time.perf_counter() - t0)
    e2e_value = job_rate(TAIL_NQ, ws, len(e2e), 1000.0 * max_over_ranks(sum(e2e), ws, "cuda"))
    dev = mhr.tails_from_device(out, TAIL_K)
    dn = n_out.cpu().numpy()
    agree = bool(np.array_equal(dn, h_n) and all(dev[q][: dn[q]].tobytes() == h_out[q][: h_n[q]].tobytes()
                                                   for q in range(TAIL_NQ)))
    if rank == 0:
        peak, peak_src = measured_peaks()
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        # fp32 add peak: 152 SMs x 128 lanes x SM clock; TransE-L1 costs one
        # subtract and one (absolute-value) add per element and pair
        n_sms = torch.cuda.get_device_properties(0).multi_processor_count
        alu_peak = n_sms * 128 * sm_mhz * 1e6 / 1e12
        flops = 2.0 * g.d * TAIL_NQ * n_cand
        achieved_alu = flops / (scan_ms / 1000.0) / 1e12
        bytes1 = g.n * g.d * eb
        achieved_hbm1 = bytes1 / (scan1 / 1000.0) / 1e9
        cpu = None
        if ws == 1 and not args.no_cpu:
            import oracle
            oracle.build()
            n = 1
            while True:
                t0 = time.perf_counter()
                oracle.tail_topk(g, H[:n], Rq[:n], TAIL_K, cand_type=TAIL_TYPE)
                dt = time.perf_counter() - t0
                if n >= TAIL_NQ or dt > 3.0:
                    break
                n = min(TAIL_NQ, n * 2)
            cpu = {"value": n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": f"first {n} of the {TAIL_NQ} heads, fp64 brute force over the type's vertices, "
                             f"OpenMP over queries, {dt:.2f} s"}
        line = {
            "metric": TAIL_METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": DATA,
            "config": {"workload": WORKLOAD_DESCS["tail"], "queries_per_step": TAIL_NQ, "K": TAIL_K,
                       "candidates": n_cand, "l2": "flushed before every call (256 MiB write, outside the events)",
                       "call": "mhr_tail_topk, synchronous; device tensors in and out"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 6 * TAIL_NQ,
                    "d2h_bytes_per_step": TAIL_NQ * TAIL_K * 16 + 4 * TAIL_NQ},
            "gpu_launches": TAIL_KERNELS_PER_CALL * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved_alu, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved_alu / alu_peak, "traffic": None,
                         "kernel": "k_tail_scan (full pass)",
                         "peak_source": f"{n_sms} SMs x 128 fp32 lanes x {sm_mhz:.0f} MHz (adds)",
                         "flops_per_launch": flops, "avg_launch_ms": scan_ms},
            "single_head": {"form": "one head against all vertices (Alg. 3)",
                            "ms_per_call": tot1 / s_steps, "scan_ms": scan1,
                            "roofline": {"bound": "hbm", "achieved": achieved_hbm1, "peak": peak, "unit": "GB/s",
                                         "frac": achieved_hbm1 / peak, "peak_source": f"{peak_src} hbm_gbs",
                                         "alg_bytes_per_launch": bytes1},
                            "work": {k: st1[k] for k in ("edges_scanned", "candidates", "rescored")}},
            "clocks": clk,
            "work_per_step": {k: st[k] for k in ("edges_scanned", "candidates", "rescored", "dense_queries")},
            "device_host_agree": agree,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    G.close()
    close_replicas(ws)
    return 0


# ------------------------------------------------------------------ beam search
BEAM_H, BEAM_K = 3, 10
BEAM_METRIC = "beam-search queries/s (Alg. 6 / Alg. 7, H=3, K=10) on 1 GB300, results identical to oracle"


def run_beam(args):
    """Beam search: CUDA events around each call (queries as host arrays of
    512 B, results copied back inside the call), L2 flushed before every call;
    roofline of the edge scoring against the fp32 add rate."""
    import torch
    import synth
    import paper_2406_07727_gb300 as mhr

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_replicas(ws, local)
    os.environ.setdefault("MHR_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "mhr_synth_cache"))
    g, S, T, _, _ = synth.workload("medium")
    S, T = rank_queries(g, S, T, rank, "medium")
    G = mhr.load_kg(g)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        mhr.mhr_beam_paths(G, S, T, BEAM_H, BEAM_K, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    st = None
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        out, n_out, st = mhr.mhr_beam_paths(G, S, T, BEAM_H, BEAM_K, stream=stream, with_stats=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tot_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), ws, "cuda")
    value = job_rate(len(S), ws, args.steps, tot_ms)
    if rank == 0:
        ms = tot_ms / args.steps
        # TransE-L1: an add, a subtract and an accumulate per element of every
        # out-edge of every held path (screened in fp32; the band near each
        # path's K-th extension rescored in fp64)
        flops = 3.0 * g.d * st["edges_scanned"]
        achieved = flops / (ms / 1000.0) / 1e12
        n_sms = torch.cuda.get_device_properties(0).multi_processor_count
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        alu_peak = n_sms * 128 * sm_mhz * 1e6 / 1e12
        cpu = None
        if ws == 1 and not args.no_cpu:
            import oracle
            oracle.build()
            n = 1
            while True:
                t0 = time.perf_counter()
                oracle.beam_paths_batch(g, S[:n], T[:n], BEAM_H, BEAM_K)
                dt = time.perf_counter() - t0
                if n >= len(S) or dt > 3.0:
                    break
                n = min(len(S), n * 2)
            cpu = {"value": n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": f"first {n} of the {len(S)} queries, fp64 beam search, OpenMP over queries, "
                             f"{dt:.2f} s"}
        line = {
            "metric": BEAM_METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": DATA,
            "config": {"workload": WORKLOAD_DESCS["beam"], "queries_per_step": len(S), "H": BEAM_H,
                       "K": BEAM_K, "l2": "flushed before every call (256 MiB write, outside the events)",
                       "call": "mhr_beam_paths, synchronous; host arrays in and out"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 8 * len(S),
                    "d2h_bytes_per_step": len(S) * BEAM_K * 64 + 4 * len(S)},
            "gpu_launches": (BEAM_H + 2) * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": None,
                         "kernel": "k_beam_level (all levels of a call)",
                         "peak_source": f"{n_sms} SMs x 128 fp32 lanes x {sm_mhz:.0f} MHz (adds)",
                         "flops_per_call": flops},
            "clocks": clk,
            "work_per_step": {"edges_scored_fp32": st["edges_scanned"], "edges_rescored_fp64": st["rescored"]},
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    G.close()
    close_replicas(ws)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import paper_2406_07727_gb300 as mhr

    g, S, T, K, spec = load_workload(rank)
    nq = len(S)
    score_fn = spec.get("score", "transe")
    G = mhr.load_kg(g, score_fn=score_fn)
    tc = 1 if score_fn == "distmult" else 0   # tensor-core middle-edge screen for DistMult
    stream = torch.cuda.current_stream()
    dS = torch.from_numpy(S.astype(np.int32)).cuda()
    dT = torch.from_numpy(T.astype(np.int32)).cuda()
    out = torch.empty((nq, K * 24), dtype=torch.uint8, device="cuda")
    n_out = torch.empty(nq, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    model, train_rep, train_s = None, None, 0.0
    if args.form == "chosen" or args.all_forms:
        t0 = time.perf_counter()
        import synth
        # training queries: the workload's own recipe on stream 3 (disjoint from the timed ones)
        if synth.WORKLOADS[WORKLOAD]["queries"] == "logdeg":
            St, Tt = synth.queries_log_degree(g, args.train_queries, seed=rank, stream=3)
        else:
            St, Tt = synth.queries_edge_biased(g, args.train_queries, seed=rank, stream=3)
        model, train_rep = mhr.train_ordering_mlp(G, St, Tt, epochs=3, batch=4096, lr=2e-3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0

    tuned = {}

    def make_opts(form):
        if form == "plain":
            o = {"prune": 0, "order": 0}
        elif form == "bound":
            o = {"prune": 1, "order": 1, "precision": tc}
        else:
            o = {"prune": 1, "order": 2, "mlp": model, "precision": tc}
        if args.chunk > 0:
            o["chunk"] = args.chunk
        elif args.chunk < 0:
            # launch shape (work-item size, scan tile) and, for DistMult, the
            # middle-edge screen from the library's autotuner, on this batch,
            # before timing
            if form not in tuned:
                to = dict(o)
                if tc and form != "plain":
                    to["precision"] = -1
                tuned[form] = mhr.mhr_autotune(G, dS, dT, K, opts=to, stream=stream)
            o["chunk"], o["tile"], o["precision"] = tuned[form][0], tuned[form][1], tuned[form][2]
        return o

    opts = make_opts(args.form)

    def step(o, with_stats=False):
        return mhr.mhr_topk_paths_batched(G, dS, dT, K, out=out, n_out=n_out, stream=stream,
                                          opts=o, with_stats=with_stats)

    dense_steps = []
    spreads = []
    expand_ms = []

    def timed(o, steps, sampler=None):
        for _ in range(args.warmup):
            step(o)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        join_ms, dev_ms, st = [], [], None
        exp_ms = []
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        # --profile-range: the headline form's timed steps form the profiler
        # range (ncu --profile-from-start off captures exactly those launches)
        prof = bool(sampler) and args.profile_range
        if prof:
            torch.cuda.profiler.start()
        # timed steps: no statistics read-back inside the timed region (it
        # synchronises after every step and is not part of the work)
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(o)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if prof:
            torch.cuda.profiler.stop()
        clk = sampler.stop() if sampler else None
        step_ms = [a.elapsed_time(b) for a, b in ev]
        el = max_over_ranks(sum(step_ms), ws, "cuda")
        if ws > 1:
            dist.barrier()
        # the library's own counters and event times, from untimed steps of the same work
        for _ in range(min(steps, 10)):
            flush.zero_()
            _, _, st = step(o, with_stats=True)
            join_ms.append(st["ms_join"])
            dev_ms.append(st["ms_device"])
            exp_ms.append(st["ms_expand"])
            dense_steps.append(st["dense_queries"])
        spreads.append(step_ms)
        expand_ms.append(statistics.mean(exp_ms))
        return el, join_ms, dev_ms, st, clk

    clocks = ClockSampler(local)
    wall0 = time.perf_counter()
    elapsed_ms, join_ms, dev_ms, stats, clk = timed(opts, args.steps, clocks)
    wall1 = time.perf_counter()
    value = job_rate(nq, ws, args.steps, elapsed_ms)
    others = {}
    for of in (["plain", "bound", "chosen"] if args.all_forms else ["plain"]):
        if of == args.form:
            continue
        o_steps = max(3, args.steps // 4)
        o_ms, o_join, o_dev, o_stats, _ = timed(make_opts(of), o_steps)
        others[of] = {"form": FORM_DESC[of], "value": job_rate(nq, ws, o_steps, o_ms),
                      "ms_per_step": o_ms / o_steps, "join_ms": statistics.mean(o_join),
                      "chunk": tuned[of][0] if of in tuned else args.chunk,
                      "tile": tuned[of][1] if of in tuned else None,
                      "middle_edge_screen": (("bf16 tensor cores" if tuned[of][2] else "fp32 CUDA cores")
                                             if of in tuned else None),
                      "work_per_step": {k: o_stats[k] for k in ("edges_scanned", "hits", "paths", "pruned_edges")}}
        if of == "plain":
            o_stats_plain = o_stats

    # end to end through the C ABI with host buffers (queries in, paths out)
    e2e_times = []
    for i in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h_out, h_n = mhr.mhr_topk_paths_batched(G, S, T, K, opts=opts)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = job_rate(nq, ws, len(e2e_times), 1000.0 * max_over_ranks(sum(e2e_times), ws, "cuda"))
    # the device run and the host run must agree bit for bit
    dev_paths = mhr.paths_from_device(out, K)
    dn = n_out.cpu().numpy()
    agree = bool(np.array_equal(dn, h_n) and all(
        dev_paths[q][: dn[q]].tobytes() == h_out[q][: h_n[q]].tobytes() for q in range(nq)))

    result = None
    if rank == 0:
        fs = frontier_stats(g, S, T)
        s_near = sum(min(f["s_f"], f["s_b"]) for f in fs)
        n_vert = sum(f["n_u"] + f["n_v"] for f in fs)
        eb = 4 if g.dtype == "f32" else 2
        plain_stats = stats if args.form == "plain" else o_stats_plain
        # algorithmic bytes of one middle-join launch (the plain method): 4 B per
        # scanned CSR entry, 2 B relation id per hit, one embedding row per
        # distinct frontier vertex
        alg_bytes = 4 * s_near + 2 * plain_stats["hits"] + eb * g.d * n_vert
        moved_bytes = 4 * stats["edges_scanned"] + 2 * stats["hits"] + eb * g.d * n_vert
        join_avg_ms = statistics.mean(join_ms)
        achieved = alg_bytes / (join_avg_ms / 1000.0) / 1e9
        peak, peak_src = measured_peaks()
        paths_per_s = plain_stats["paths"] * ws * args.steps / (elapsed_ms / 1000.0)
        cpu, parity, perr = None, None, None
        if ws == 1 and not args.no_cpu:
            cpu, sample = cpu_oracle_rate(g, S, T, K, fn=score_fn)
            parity = oracle_parity(h_out, h_n, sample)
        perr = precision_error(mhr, G, S, T, h_out, h_n)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": DATA,
            "config": {"workload": WORKLOAD_DESC, "queries_per_step": nq, "K": K,
                       "score_fn": score_fn, "form": FORM_DESC[args.form],
                       "middle_edge_screen": ("bf16 tensor cores (hi/lo split)" if opts.get("precision") == 1
                                              else "fp32 CUDA cores"),
                       "l2": "flushed before every step (256 MiB write, excluded from the step time)",
                       "parallelism": "replicas (each rank its own queries)" if ws > 1 else "single GPU",
                       "launch": "three CUDA graphs per step (before / join / after)",
                       "chunk": opts.get("chunk", "library default"),
                       "tile": opts.get("tile", "library default"),
                       "autotune_ms": ({f"{'tc' if p else 'fp32'}/{c}x{t}": v
                                        for (p, c, t), v in tuned[args.form][3].items()}
                                       if args.form in tuned else None)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * nq,
                    "d2h_bytes_per_step": nq * K * 24 + 4 * nq},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": TRAFFIC_NCU.get((WORKLOAD, args.form, opts.get("chunk"), opts.get("tile"))),
                         "traffic_scope": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the main join launch",
                         "kernel": "k_middle (middle join)", "peak_source": f"{peak_src} hbm_gbs",
                         "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": join_avg_ms,
                         "bytes_moved_per_launch": moved_bytes,
                         "note": "achieved credits the plain method's algorithmic bytes (effective rate for the pruned form)"},
            "clocks": clk,
            "scored_paths_per_s": paths_per_s,
            "work_per_step": {"edges_scanned": stats["edges_scanned"], "edges_scanned_plain": s_near,
                              "hits": stats["hits"], "paths": stats["paths"],
                              "pruned_edges": stats["pruned_edges"],
                              "candidates": stats["candidates"], "rescored": stats["rescored"],
                              "dense_queries": stats["dense_queries"]},
            "other_forms": others,
            "learned_order": ({"train_queries": args.train_queries, "rows": train_rep.rows,
                               "loss_first": train_rep.loss_first, "loss_last": train_rep.loss_last,
                               "train_s": train_s} if train_rep else None),
            "device_ms_per_step": statistics.mean(dev_ms),
            "step_ms_spread": {"min": min(spreads[0]), "median": statistics.median(spreads[0]),
                               "max": max(spreads[0])},
            "device_ms_spread": {"min": min(dev_ms), "median": statistics.median(dev_ms), "max": max(dev_ms)},
            "join_ms_spread": {"min": min(join_ms), "median": statistics.median(join_ms), "max": max(join_ms)},
            "steps_with_dense_queries": sum(1 for x in dense_steps if x),
            "stats_steps": "work counters, device/join times and dense counts come from up to 10 untimed "
                           "steps of the same work after the timed loop",
            "device_host_agree": agree,
            "wall_s_timed_loop": wall1 - wall0,
        }
        if cpu is not None:
            result["cpu_baseline"] = cpu
            result["oracle_parity"] = parity
        result["precision_error"] = perr
        # hop-1 / hop-3 expansion (a2, a3): CSR entries of the rows of s and t
        # plus one embedding row per distinct frontier vertex, per launch
        slots = sum(f["deg_s"] + f["deg_t"] for f in fs)
        x_bytes = slots * (4 + 2) + eb * g.d * (n_vert + 2 * nq)
        x_ms = expand_ms[0]
        result["expansion_roofline"] = {
            "bound": "hbm", "kernel": "k_expand (hop-1 / hop-3 expansion)",
            "achieved": x_bytes / (x_ms / 1000.0) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": x_bytes / (x_ms / 1000.0) / 1e9 / peak, "alg_bytes_per_launch": x_bytes,
            "bytes_loaded_per_launch": slots * (4 + 2 + eb * g.d), "avg_launch_ms": x_ms,
            "peak_source": f"{peak_src} hbm_gbs"}
        # the forms side by side (all return identical results)
        rates = {args.form: value}
        rates.update({k: v["value"] for k, v in others.items()})
        result["form_comparison"] = {
            "queries_per_s": rates,
            "fastest": max(rates, key=rates.get),
            "headline_vs_plain": (value / rates["plain"]) if "plain" in rates and args.form != "plain" else None,
            "headline_vs_bound": (value / rates["bound"]) if "bound" in rates and args.form != "bound" else None}
        print(json.dumps(result), flush=True)
    G.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--chunk", type=int, default=-1,
                    help="middle-join work item size (-1 = autotuned before timing, 0 = library default)")
    ap.add_argument("--workload", default="batching", choices=sorted(WORKLOAD_DESCS),
                    help="batching is the benchmark workload; the others are extra measurements")
    ap.add_argument("--all-forms", type=int, default=1, help="also time the other forms (plain, bound, chosen)")
    ap.add_argument("--train-queries", type=int, default=20000)
    ap.add_argument("--K", type=int, default=0, help="override the workload's K (e.g. 500 for the learned workload)")
    ap.add_argument("--profile-range", action="store_true",
                    help="wrap the headline form's timed steps in a CUDA profiler range")
    ap.add_argument("--form", default="chosen", choices=["plain", "bound", "chosen"],
                    help="plain: every hit scored; chosen: provable bound pruning (same output)")
    args = ap.parse_args()
    global WORKLOAD, WORKLOAD_DESC, K_OVERRIDE
    WORKLOAD, WORKLOAD_DESC = args.workload, WORKLOAD_DESCS[args.workload]
    K_OVERRIDE = args.K
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "tail":
        return run_tail(args)
    if args.workload == "beam":
        return run_beam(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
