#!/usr/bin/env python3
"""Benchmark of the frontier SSSP hot path on one or more B300 GPUs.

Default workload (the headline): single-source SSSP on the RMAT scale-22
graph (edge factor 16, a,b,c,d = .57,.19,.19,.05, symmetrised,
deduplicated, no self-loops, uint32 weights U[1,255] from seed 1), source =
highest-degree vertex, bulk-synchronous CUDA-graph loop with the library's
defaults (light/heavy buckets, warp-streaming push).

One step = one gg_sssp call (distance init through convergence) with the
graph resident in HBM.  value = GTEPS = m_trav / step time, m_trav = sum of
out-degrees of the reached vertices (each edge of the reached component once).

Every timed result is checked before a line is printed: the distance vector
(and the batched matrix, and every served query's vector) must hash to the
value tests/golden/workloads.json stores for it, which tests/golden/
make_golden.py wrote from the CPU oracle.  A mismatch prints no line and
exits 1.

Sub-objects of the line: rmat20 (single source on RMAT scale 20), grid4096
(the 4096^2 high-diameter grid under the CUDA-graph loop, the persistent
cooperative kernel and the asynchronous work queue), batched (64 seeded
sources on RMAT-22 in one fused loop vs back-to-back gg_sssp) and serving
(the 2,000-query Poisson stream over the 32-graph pool).

Multi-GPU (torchrun): single-source SSSP does not shard, so every rank runs
an independent replica of the same workload ("replicas only"); value = edges
traversed by all ranks / max-over-ranks time.  No collective touches the data
path; ranks only meet at the timing barriers.

--impl reference: the CPU oracle (binary-heap Dijkstra) on the same workload,
on the host cores, printed on the same JSON schema.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SSSP GTEPS & %HBM roofline (1 B300); batched queries/s + p50/p99 vs single-source"
L2_BYTES = 126 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gg", choices=["gg", "reference"])
    p.add_argument("--workload", default="rmat22")
    p.add_argument("--policy", default="graph", choices=["graph", "async", "host", "persistent"])
    p.add_argument("--direction", default="push", choices=["auto", "push", "pull"])
    p.add_argument("--lb", default="auto", choices=["auto", "mp", "bins", "warp", "local"])
    p.add_argument("--batch-scale", type=int, default=22, help="RMAT scale of the batched run (22 = the workload)")
    p.add_argument("--batch-policy", default="graph", choices=["graph", "host"],
                   help="host: supersteps launched one by one (for profilers)")
    p.add_argument("--delta", type=int, default=0, help="near-far bucket width (0 = graph default, -1 = none)")
    p.add_argument("--alpha", type=int, default=0)
    p.add_argument("--beta", type=int, default=0)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the batched 64-source RMAT-22 measurement")
    p.add_argument("--no-serve", action="store_true", help="skip the 32-graph serving measurement")
    p.add_argument("--serve-queries", type=int, default=2000)
    p.add_argument("--no-rmat20", action="store_true", help="skip the RMAT-20 single-source sub-line")
    p.add_argument("--no-grid", action="store_true", help="skip the 4096^2 grid policy comparison")
    p.add_argument("--batch-trace", default="",
                   help="write the batched run's per-superstep trace (kind, entries, edges, next size) to this file")
    p.add_argument("--trace", default="",
                   help="write the single-source stats run's per-superstep trace (frontier size, frontier edges, "
                        "kind, next frontier size) to this file")
    p.add_argument("--ref-seconds", type=float, default=240.0,
                   help="--impl reference: stop adding steps once this much host time is spent")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


L2_FLUSH_BYTES = 512 << 20   # > the B300's 126 MB L2
GRAPH_LOOP_UNROLL = 8        # superstep kernels per iteration of the library's CUDA-graph loop
NOMINAL_HBM_GBS = 8000.0     # the nominal HBM3e figure the 35 % target was also stated against (context only)


def kernel_source_hash() -> str:
    """sha256 of the superstep kernel's sources: a stored DRAM-traffic figure
    is reported only while the kernel it was measured on is unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in ("gg_bsp.cu", "gg_common.cuh", "gg_host.h"):
        with open(os.path.join(ROOT, "paper_2212_08200_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_traffic(workload: str, direction: str, lb: str, delta: int):
    """DRAM bytes (read + write) of the superstep kernel over one whole SSSP,
    from the ncu capture summarised in profiles/k_superstep_traffic.json, when
    that capture matches this workload, these options and the current kernel
    source; otherwise None."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_superstep_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    for e in d.get("captures", []):
        if (e.get("workload") == workload and e.get("direction") == direction and e.get("lb") == lb
                and e.get("delta") == delta and e.get("source_sha256") == kernel_source_hash()):
            return float(e["dram_bytes_per_sssp"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(n, m_trav, n_reach):
    """Per SSSP: 12 B per traversed edge (col 4 + weight 4 + dist[dst] 4),
    20 B per reached vertex (2 row offsets 8 + dist[u] 4 + frontier write 4 +
    frontier read 4), 4 B per vertex for the distance write."""
    return 12 * m_trav + 20 * n_reach + 4 * n, 12 * m_trav + 20 * n_reach


def cpu_baseline(ro, col, w, src, seconds):
    import oracle
    times = []
    t_end = time.perf_counter() + seconds
    d = None
    while time.perf_counter() < t_end or not times:
        t0 = time.perf_counter()
        d = oracle.dijkstra(ro, col, w, src)
        times.append(time.perf_counter() - t0)
        if len(times) >= 50:
            break
    m_trav = oracle.traversed_edges(ro, d)
    t = statistics.median(times)
    return {"value": m_trav / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} full single-source binary-heap Dijkstra runs on the same graph and source "
                      f"(median {t * 1e3:.1f} ms each, 1 host thread)"}


def cpu_baseline_batch(ro, col, w, srcs):
    """The oracle's multi-source Dijkstra (one source per host thread) on a
    bounded sample of the batch's sources: as many sources as host threads, at
    most all of them, timed as one wall-clock run."""
    import oracle
    t = max(1, min(len(srcs), os.cpu_count() or 1))
    t0 = time.perf_counter()
    oracle.dijkstra_many(ro, col, w, np.asarray(srcs[:t], np.uint32), threads=t)
    dt = time.perf_counter() - t0
    return {"queries_per_s": t / dt, "cores": t, "kind": "oracle",
            "sample": f"the first {t} of the {len(srcs)} sources, one binary-heap Dijkstra per host thread "
                      f"({dt:.2f} s wall)"}


def cpu_baseline_queries(queries, total):
    """The oracle's Dijkstra over a bounded sample of served queries (graph
    CSR, source), one query per host thread at a time (the ctypes call
    releases the GIL): twice as many queries as host threads, at most all."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    t = max(1, os.cpu_count() or 1)
    sample = queries[:2 * t]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(t) as ex:
        list(ex.map(lambda q: oracle.dijkstra(*q), sample))
    dt = time.perf_counter() - t0
    return {"queries_per_s": len(sample) / dt, "cores": min(t, len(sample)), "kind": "oracle",
            "sample": f"the first {len(sample)} of the {total} queries, binary-heap Dijkstra on {t} host threads "
                      f"({dt:.2f} s wall)"}


def shard(items, rank, world):
    """This rank's share of a work list: items rank, rank + world, ...
    (disjoint across ranks, together complete)."""
    return items[rank::world]


def reduce_over_ranks(value, op, pg):
    """max / sum of a per-rank float over all ranks (identity without a
    process group).  Timing only: no data-path collective."""
    if pg is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() and pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX if op == "max" else pg.ReduceOp.SUM)
    return float(t.item())


def golden():
    """The stored oracle results (tests/golden/workloads.json, written by
    tests/golden/make_golden.py from the CPU oracle); {} when absent."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def sha256_u32(a) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a, np.uint32).tobytes()).hexdigest()


class NotVerified(RuntimeError):
    """A timed result differs from the stored oracle result: no line is printed."""


def verify_single(name: str, dist_host) -> bool | None:
    """True when the distances hash to the stored oracle hash of workload
    `name`, None when no hash is stored for it; raises NotVerified on a
    mismatch."""
    rec = golden().get(name)
    if not rec or "dist_sha256" not in rec:
        return None
    if sha256_u32(dist_host) != rec["dist_sha256"]:
        raise NotVerified(f"{name}: the distances differ from the oracle's (stored sha256 {rec['dist_sha256'][:16]})")
    return True


def time_sssp(gg, torch, g, src, opts, stream, steps, warmup, flush):
    """Per-step milliseconds of gg_sssp_ex(src) with the L2 flushed (flush
    buffer written outside the events) before every timed step."""
    dist_t = torch.empty(g.n, dtype=torch.uint32, device="cuda")
    for _ in range(max(warmup, 1)):
        gg.gg_sssp_ex(g.handle, src, dist_t, opts, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        gg.gg_sssp_ex(g.handle, src, dist_t, opts, stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    g.check()
    return [a.elapsed_time(b) for a, b in ev]


def stats_run(gg, torch, g, src, policy, stream, **kw):
    """One SSSP with statistics; (distances on the host, stats dict)."""
    st = gg.gg_stats()
    dist_t = torch.empty(g.n, dtype=torch.uint32, device="cuda")
    gg.gg_sssp_ex(g.handle, src, dist_t, gg.make_options(policy=policy, stats=st, **kw), stream)
    torch.cuda.synchronize()
    g.check()
    return dist_t.cpu().numpy(), st.as_dict()


def run_rmat20(gg, torch, stream, flush, steps=10):
    """Single source on RMAT scale 20 from the hub with the library defaults
    (the smaller RMAT workload), verified against the stored oracle hash."""
    import graphgen
    ro, col, w, src = graphgen.workload("rmat20")
    g = gg.Graph(ro, col, w, symmetric=True, stream=stream)
    d, st = stats_run(gg, torch, g, src, gg.GG_POLICY_BSP_GRAPH, stream, direction=gg.GG_DIR_PUSH)
    ok = verify_single("rmat20", d)
    reach = d != gg.GG_INF
    n, m_trav, n_reach = g.n, int(np.diff(ro.astype(np.int64))[reach].sum()), int(reach.sum())
    per = time_sssp(gg, torch, g, src, gg.make_options(direction=gg.GG_DIR_PUSH), stream, steps, 3, flush)
    g.close()
    t = statistics.median(per)
    hbm, peak_kind = peaks()
    b_all, _ = algorithmic_bytes(n, m_trav, n_reach)
    return {"workload": workload_desc("rmat20"), "source": int(src), "ms": t, "ms_min": min(per),
            "GTEPS": m_trav / (t * 1e-3) / 1e9, "m_trav": m_trav, "n_reach": n_reach, "algorithmic_bytes": b_all,
            "roofline_frac": b_all / (t * 1e-3) / 1e9 / hbm, "peak_GBs": hbm, "peak_kind": peak_kind,
            "supersteps": st["iterations"], "edges_scanned": st["edges_scanned"], "verified": ok,
            "l2": "flushed before every timed run", "runs": len(per)}


def run_grid4096(gg, torch, stream, flush, steps=3):
    """The 4096^2 grid (16.7 M vertices, 67 M edges, weights U[1,1000]) from
    the corner under the paper's two timing models: bulk-synchronous
    supersteps (CUDA-graph loop with the library's defaults, which on this
    low-degree graph include warp-local rounds; the same loop without them;
    the persistent cooperative kernel) and the asynchronous persistent kernel
    over a device work queue; each verified against the stored oracle hash."""
    import graphgen
    ro, col, w, src = graphgen.workload("grid4096")
    g = gg.Graph(ro, col, w, symmetric=True, stream=stream)
    m_trav = int(col.shape[0])
    out = {"workload": workload_desc("grid4096"), "source": int(src), "n": g.n, "m": g.m, "m_trav": m_trav}
    for name, pol, lb in (("bsp_cuda_graph", gg.GG_POLICY_BSP_GRAPH, gg.GG_LB_AUTO),
                          ("bsp_cuda_graph_no_local_rounds", gg.GG_POLICY_BSP_GRAPH, gg.GG_LB_WARP),
                          ("bsp_persistent", gg.GG_POLICY_BSP_PERSISTENT, gg.GG_LB_AUTO),
                          ("async_queue", gg.GG_POLICY_ASYNC_PERSISTENT, gg.GG_LB_AUTO)):
        d, st = stats_run(gg, torch, g, src, pol, stream, direction=gg.GG_DIR_PUSH, lb_mode=lb)
        ok = verify_single("grid4096", d)
        per = time_sssp(gg, torch, g, src, gg.make_options(policy=pol, direction=gg.GG_DIR_PUSH, lb_mode=lb), stream,
                        steps, 1, flush)
        t = statistics.median(per)
        out[name] = {"ms": t, "ms_min": min(per), "GTEPS": m_trav / (t * 1e-3) / 1e9,
                     "supersteps": st["iterations"], "edges_scanned": st["edges_scanned"],
                     "edges_scanned_per_m_trav": st["edges_scanned"] / m_trav, "verified": ok, "runs": len(per)}
    g.close()
    out["async_vs_bsp"] = out["async_queue"]["ms"] / out["bsp_cuda_graph"]["ms"]
    return out


def run_batched(gg, torch, k=64, seed=1, scale=22, policy="graph", cpu_sample=True, graph=None, trace_file=""):
    """Batched multi-source SSSP on RMAT-22 (64 seeded sources, one fused
    launch sequence) vs the same 64 sources as back-to-back gg_sssp calls.
    The whole distance matrix is checked against the stored oracle hash.
    scale / policy other than 22 / graph serve profiling (ncu cannot see the
    kernels inside the CUDA-graph loop; "host" launches them one by one)."""
    import graphgen
    pol = {"graph": gg.GG_POLICY_BSP_GRAPH, "host": gg.GG_POLICY_BSP_HOST}[policy]
    ro, col, w = graph if graph is not None else graphgen.rmat(scale, 16, seed=1, W=255)
    srcs = graphgen.sample_sources(ro, k, seed=seed)
    g = gg.Graph(ro, col, w, symmetric=True)
    n = g.n
    out = torch.empty(n * k, dtype=torch.uint32, device="cuda")
    single = torch.empty(n, dtype=torch.uint32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = gg.gg_stats()
    trace = torch.zeros(4 * 65536, dtype=torch.uint32, device="cuda") if trace_file else None
    g.sssp_batch(srcs, out, stats=st, policy=pol, **({"trace": trace, "trace_cap": 65536} if trace_file else {}))
    g.check()
    if trace_file:
        np.savetxt(trace_file, trace.cpu().numpy().reshape(-1, 4)[:min(st.iterations, 65536)], fmt="%d",
                   header="kind (0 light, 1 split, 2 heavy push, 3 mask clear, 4 heavy pull, 5 heavy pull that ends the buckets; +16 after bucketing) "
                          "entries edges next_frontier")
    rec = golden().get(f"rmat{scale}_batch{k}")
    verified = None
    if rec and seed == 1 and [int(x) for x in srcs] == rec["sources"]:
        host = out.cpu().numpy()
        if sha256_u32(host) != rec["matrix_sha256"]:
            bad = [s for s in range(k) if sha256_u32(host.reshape(n, k)[:, s]) != rec["column_sha256"][s]]
            raise NotVerified(f"batched RMAT-{scale} x {k}: columns {bad[:8]} differ from the oracle's")
        verified = True
        m_trav_all = int(sum(rec["m_trav"]))
        del host
    else:
        m_trav_all = None
    tb = []
    for _ in range(3):
        e0.record()
        g.sssp_batch(srcs, out, policy=pol)
        e1.record()
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1))
    for s_ in srcs[:4]:
        g.sssp(int(s_), single)
    torch.cuda.synchronize()
    e0.record()
    for s_ in srcs:
        g.sssp(int(s_), single)
    e1.record()
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1)
    g.check()
    g.close()
    t = statistics.median(tb)
    cpu = cpu_baseline_batch(ro, col, w, srcs) if cpu_sample else None
    return {"workload": f"RMAT scale {scale} EF16, {k} seeded sources (splitmix64 seed {seed}), "
                        f"dist matrix {n} x {k} u32",
            "policy": policy,
            "queries_per_s": k / t * 1e3, "ms": t, "ms_all": tb, "back_to_back_queries_per_s": k / t1 * 1e3,
            "back_to_back_ms": t1, "speedup": t1 / t, "supersteps": st.iterations,
            "edges_scanned": st.edges_scanned,
            "gteps_aggregate": (m_trav_all / (t * 1e-3) / 1e9) if m_trav_all else None,
            "verified": verified, "cpu_baseline": cpu,
            "l2": "not flushed: every run's working set (0.5 GB of edges, the 1 GiB distance matrix) exceeds the "
                  "126 MB L2"}


def run_serving(gg, torch, nq=2000, seed=1, cpu_sample=True):
    """Poisson stream of (graph, source) queries over the 32-graph pool into
    the continuous-batching server, at saturation (all queued at t=0) and at
    50 % / 90 % of the saturation rate; vs the same queries back to back.
    Every query's distances are checked against the stored oracle hash after
    the saturation pass and after the back-to-back pass."""
    import graphgen
    pool = [graphgen.build_pool_graph(e) for e in graphgen.serving_pool_spec()]
    graphs = [gg.Graph(ro, col, w, symmetric=True) for ro, col, w in pool]
    degs = [np.diff(ro.astype(np.int64)) for ro, _, _ in pool]
    gids, srcs, _ = graphgen.poisson_queries(degs, nq, seed=seed)
    outs = [torch.empty(graphs[gi].n, dtype=torch.uint32, device="cuda") for gi in gids]
    maxn = max(gr.n for gr in graphs)
    srv = gg.Server(max_graph_vertices=maxn, max_slots=64, supersteps_per_launch=8)
    rec = golden().get("serving_pool")
    checkable = (rec is not None and rec["seed"] == seed and rec["queries"] == nq
                 and rec["graph"] == [int(x) for x in gids] and rec["source"] == [int(x) for x in srcs])

    def verify(what):
        if not checkable:
            return None
        bad = []
        for i in range(nq):
            if sha256_u32(outs[i].cpu().numpy())[:16] != rec["dist_sha256_16"][i]:
                bad.append(i)
        if bad:
            raise NotVerified(f"serving ({what}): queries {bad[:8]} ({len(bad)} in all) differ from the oracle's")
        return True

    def stream(rate):
        _, _, arr = graphgen.poisson_queries(degs, nq, seed=seed, rate_qps=rate)
        for o in outs:
            o.view(torch.int32).fill_(0x5A5A5A5A)   # a query that writes nothing cannot pass the check
        torch.cuda.synchronize()
        srv.reset_stats()
        t0 = time.perf_counter()
        ts = []
        for i in range(nq):
            if rate is not None:
                delay = arr[i] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            ts.append(srv.submit(graphs[gids[i]], int(srcs[i]), outs[i]))
        bad = sum(1 for t in ts if srv.wait(t, 600000) != 0)
        dt = time.perf_counter() - t0
        st = srv.stats()
        return {"queries_per_s": nq / dt, "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                "max_in_flight": st["max_running"], "launches": st["launches"], "failed": bad}

    stream(None)                       # warm-up pass
    sat = stream(None)
    verified = verify("saturation")
    loads = {}
    for frac in (0.5, 0.9):
        loads[f"{int(frac * 100)}pct"] = stream(sat["queries_per_s"] * frac)
    srv.close()
    # back to back: the same queries through gg_sssp, one after another on one stream
    for o in outs:
        o.view(torch.int32).fill_(0x5A5A5A5A)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(nq):
        graphs[gids[i]].sssp(int(srcs[i]), outs[i])
    torch.cuda.synchronize()
    b2b = nq / (time.perf_counter() - t0)
    verified_b2b = verify("back to back")
    for gr in graphs:
        gr.close()
    cpu = (cpu_baseline_queries([(*pool[gids[i]], int(srcs[i])) for i in range(nq)], nq)
           if cpu_sample else None)
    return {"workload": "32-graph pool (RMAT scales 12-20 EF 8/16, grids 64^2-2048^2, U[1,255]), "
                        f"{nq} queries, graph uniform, source uniform over degree>=1, Poisson seed {seed}",
            "saturation": sat, "load": loads, "back_to_back_queries_per_s": b2b,
            "speedup": sat["queries_per_s"] / b2b, "verified": verified, "verified_back_to_back": verified_b2b,
            "cpu_baseline": cpu}


def workload_desc(name):
    import graphgen
    return graphgen.WORKLOADS.get(name, name)


def run_reference(args):
    """The CPU oracle (single-thread binary-heap Dijkstra) on the workload:
    W warm-up and K timed steps, each one full SSSP, cut short (and said so)
    once --ref-seconds of host time are spent."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import graphgen
    import oracle
    ro, col, w, src = graphgen.workload(args.workload)
    budget = max(args.ref_seconds, 1.0)
    t_begin = time.perf_counter()
    warm = 0
    for _ in range(args.warmup):
        if warm and time.perf_counter() - t_begin > budget / 4:
            break
        oracle.dijkstra(ro, col, w, src)
        warm += 1
    steps = []
    d = None
    while len(steps) < args.steps and (time.perf_counter() - t_begin < budget or not steps):
        t0 = time.perf_counter()
        d = oracle.dijkstra(ro, col, w, src)
        steps.append(time.perf_counter() - t0)
    m_trav = oracle.traversed_edges(ro, d)
    t = statistics.median(steps)
    val = m_trav / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": args.gpus,
            "device": "host CPU, 1 thread (the oracle uses no GPU)",
            "steps": len(steps), "warmup": warm, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload), "n": int(ro.shape[0] - 1), "m": int(col.shape[0]),
                       "source": int(src), "m_trav": m_trav},
            "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{len(steps)} of {args.steps} requested steps after {warm} warm-up runs, "
                                       f"each a full single-source binary-heap Dijkstra on the host "
                                       f"(bounded to ~{budget:.0f} s in all)"},
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    try:
        run_gg(args)
    except NotVerified as e:
        print(f"bench: result check failed, no line printed: {e}", file=sys.stderr, flush=True)
        sys.exit(1)


def run_gg(args):
    import torch

    import graphgen
    import paper_2212_08200_b300 as gg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    gg.load()
    ro, col, w, src = graphgen.workload(args.workload)
    n, m = int(ro.shape[0] - 1), int(col.shape[0])
    policy = {"graph": gg.GG_POLICY_BSP_GRAPH, "async": gg.GG_POLICY_ASYNC_PERSISTENT,
              "host": gg.GG_POLICY_BSP_HOST, "persistent": gg.GG_POLICY_BSP_PERSISTENT}[args.policy]
    direction = {"auto": gg.GG_DIR_AUTO, "push": gg.GG_DIR_PUSH, "pull": gg.GG_DIR_PULL}[args.direction]
    stream = torch.cuda.current_stream()
    g = gg.Graph(ro, col, w, symmetric=True, stream=stream)
    dist_t = torch.empty(n, dtype=torch.uint32, device="cuda")
    lb = {"auto": gg.GG_LB_AUTO, "mp": gg.GG_LB_MERGE_PATH, "bins": gg.GG_LB_BINS, "warp": gg.GG_LB_WARP,
          "local": gg.GG_LB_LOCAL}[args.lb]
    delta = gg.GG_DELTA_NONE if args.delta < 0 else args.delta
    opts = gg.make_options(policy=policy, direction=direction, lb_mode=lb, pull_alpha=args.alpha, pull_beta=args.beta,
                           delta=delta)

    def step():
        gg.gg_sssp_ex(g.handle, src, dist_t, opts, stream)

    # correctness of what is timed: a stats run whose distances must hash to
    # the stored oracle hash of this workload (no line is printed otherwise)
    st = gg.gg_stats()
    trace = torch.zeros(4 * 65536, dtype=torch.uint32, device="cuda") if args.trace else None
    torch.cuda.nvtx.range_push("gg_sssp_stats_run")   # lets a profiler select exactly one SSSP's launches
    gg.gg_sssp_ex(g.handle, src, dist_t, gg.make_options(policy=policy, direction=direction, lb_mode=lb,
                                                         pull_alpha=args.alpha, pull_beta=args.beta, stats=st,
                                                         delta=delta,
                                                         **({"trace": trace, "trace_cap": 65536} if args.trace
                                                            else {})), stream)
    torch.cuda.nvtx.range_pop()
    g.check()
    if args.trace:
        np.savetxt(args.trace, trace.cpu().numpy().reshape(-1, 4)[:min(st.iterations, 65536)], fmt="%d",
                   header="frontier size, frontier edges, kind (0 push, 1 pull, 2 split, 3 heavy push, "
                          "4 heavy pull, 5 heavy pull that ends the buckets), next frontier size")
    d_host = dist_t.cpu().numpy()
    verified = verify_single(args.workload, d_host)
    reach = d_host != gg.GG_INF
    m_trav = int(np.diff(ro.astype(np.int64))[reach].sum())
    n_reach = int(reach.sum())
    stats = st.as_dict()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # fixed per-call cost: init kernels + graph launch + one single-vertex superstep
    fixed_opts = gg.make_options(policy=policy, direction=gg.GG_DIR_PUSH, max_iterations=1, delta=gg.GG_DELTA_NONE)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    fixed_src = src
    if policy == gg.GG_POLICY_ASYNC_PERSISTENT:
        # the async kernel has no superstep cap: its fixed cost is a run from a
        # vertex without out-edges (init + seed + a kernel that finds no work)
        iso = np.flatnonzero(np.diff(ro.astype(np.int64)) == 0)
        fixed_src = int(iso[0]) if iso.size else None
    fixed = []
    for _ in range(5 if fixed_src is not None else 0):
        ev[0].record(stream)
        gg.gg_sssp_ex(g.handle, fixed_src, dist_t, fixed_opts, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        fixed.append(ev[0].elapsed_time(ev[1]))
    t_fixed_ms = statistics.median(fixed) if fixed else 0.0
    step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # L2 (126 MB) is flushed before every timed step by writing a larger
    # buffer, outside the step's events: no step starts with a warm cache
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    for k in range(args.steps):
        flush.fill_(k)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(per) / args.steps
    # the last timed step's distances must be the verified ones too
    g.check()
    if verified and sha256_u32(dist_t.cpu().numpy()) != sha256_u32(d_host):
        raise NotVerified("the last timed step's distances differ from the verified stats run's")
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = world * m_trav / (ms * 1e-3) / 1e9

    hbm, peak_kind = peaks()
    b_all, b_super = algorithmic_bytes(n, m_trav, n_reach)
    super_ms = max(statistics.median(per) - t_fixed_ms, 1e-6)
    achieved = b_super / (super_ms * 1e-3) / 1e9
    iters = stats["iterations"]
    # init + init tail + the supersteps; the CUDA-graph loop runs its superstep
    # kernel in groups of GRAPH_LOOP_UNROLL per evaluation of the loop condition
    # (those past the last superstep return at once but are launches too)
    launches_per_step = 2 + iters
    if policy == gg.GG_POLICY_BSP_GRAPH:
        launches_per_step = 2 + -(-iters // GRAPH_LOOP_UNROLL) * GRAPH_LOOP_UNROLL
    if policy == gg.GG_POLICY_ASYNC_PERSISTENT:
        launches_per_step = 3   # init, seed, persistent kernel (plus one memset node)
    elif policy == gg.GG_POLICY_BSP_PERSISTENT:
        launches_per_step = 3   # init, init tail, persistent superstep kernel

    # end to end through the public API with host buffers: upload the CSR from
    # pinned memory, run, read the distances back, free the handle
    e2e = None
    if not args.no_e2e:
        pin = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in (ro, col, w)]
        arrs = [p.numpy().view(np.uint32) for p in pin]
        out_h = torch.empty(n, dtype=torch.int32).pin_memory()
        k2 = max(3, min(args.steps, 10))
        for it in range(k2 + 1):
            if it == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            h = gg.gg_graph_create_csr(arrs[0], arrs[1], arrs[2], symmetric=True, stream=stream)
            gg.gg_sssp_ex(h, src, dist_t, opts, stream)   # the timed path's options
            out_h.copy_(dist_t.view(torch.int32), non_blocking=True)
            torch.cuda.synchronize()
            gg.gg_graph_destroy(h)
        e2e_s = (time.perf_counter() - t0) / k2
        if verified and sha256_u32(out_h.numpy().view(np.uint32)) != sha256_u32(d_host):
            raise NotVerified("the end-to-end run's distances differ from the oracle's")
        e2e = {"value": world * m_trav / e2e_s / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": 4 * (n + 1) + 8 * m, "d2h_bytes_per_step": 4 * n,
               "ms_per_step": e2e_s * 1e3,
               "what": "gg_graph_create_csr from pinned host CSR + gg_sssp_ex + distances copied to pinned host "
                       "+ gg_graph_destroy, wall clock"}

    # sub-lines: the smaller RMAT and the high-diameter grid (timing models)
    rmat20 = grid = None
    if not args.no_rmat20:
        rmat20 = run_rmat20(gg, torch, stream, flush)
    if not args.no_grid:
        grid = run_grid4096(gg, torch, stream, flush)
    del flush

    # batched and served queries shard naturally: every rank runs its own
    # seeded stream (per-GPU work fixed) and the queries/s add up
    batched = serving = None
    cpu_sample = rank == 0 and world == 1 and not args.no_cpu_baseline   # oracle baselines: rank 0 at N=1
    if not args.no_batch:
        same = args.workload == f"rmat{args.batch_scale}"
        g.close()    # the batch builds its own handle (the headline's is no longer needed)
        batched = run_batched(gg, torch, seed=1 + rank, scale=args.batch_scale, policy=args.batch_policy,
                              cpu_sample=cpu_sample, graph=(ro, col, w) if same else None,
                              trace_file=args.batch_trace if rank == 0 else "")
        batched["queries_per_s_all_ranks"] = reduce_over_ranks(batched["queries_per_s"], "sum", pg)
    if not args.no_serve:
        serving = run_serving(gg, torch, args.serve_queries, seed=1 + rank, cpu_sample=cpu_sample)
        serving["queries_per_s_all_ranks"] = reduce_over_ranks(serving["saturation"]["queries_per_s"], "sum", pg)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ro, col, w, src, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "verified": verified,
            "config": {"workload": workload_desc(args.workload), "n": n, "m": m, "source": int(src),
                       "m_trav": m_trav, "n_reach": n_reach, "policy": args.policy, "direction": args.direction,
                       "lb": args.lb, "delta": args.delta,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"L2 flushed before every timed step ({L2_FLUSH_BYTES >> 20} MiB written outside "
                             f"the step's events); dist re-initialised every step",
                       "verified_against": "sha256 of the stats run's and the last timed step's distances = the "
                                           "oracle's stored hash (tests/golden/workloads.json)",
                       "supersteps": iters, "pull_supersteps": stats["pull_iterations"],
                       "edges_scanned": stats["edges_scanned"], "step_ms_min": min(per), "step_ms_max": max(per),
                       "step_ms_median": statistics.median(per)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "traffic": kernel_traffic(args.workload, args.direction, args.lb, args.delta),
                         "traffic_unit": "DRAM bytes per SSSP (all supersteps), ncu, cold L2",
                         "peak_kind": peak_kind,
                         "kernel": ("k_async (the whole run)" if policy == gg.GG_POLICY_ASYNC_PERSISTENT else
                                    "k_bsp_persistent (all supersteps)" if policy == gg.GG_POLICY_BSP_PERSISTENT else
                                    "k_superstep (all supersteps of one SSSP)"),
                         "algorithmic_bytes": b_super, "kernel_ms": super_ms, "fixed_ms": t_fixed_ms,
                         "whole_step_frac": b_all / (ms * 1e-3) / 1e9 / hbm,
                         "frac_nominal_8tbs": achieved / NOMINAL_HBM_GBS},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "rmat20": rmat20,
            "grid4096": grid,
            "batched": batched,
            "serving": serving,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "gpu": torch.cuda.get_device_name(),
        }
        print(json.dumps(line), flush=True)
    if args.no_batch:
        g.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
