"""Benchmark of the LSH-MF hot path on GB300.

A step is one whole training job on the Netflix-shaped workload
(480k users x 17,770 items, 100M ratings, F = K = 64, L = 16 tables x 12 bits,
10 epochs): COO -> CSC, simLSH neighbour build (signatures, buckets, top-K),
training layout with the explicit-neighbour index, 10 stratified SGD epochs,
held-out RMSE.  `value` = rating-updates/s = epochs * nnz_train / step time,
inputs resident in HBM.  `e2e` = the same with the inputs copied from pinned
host memory inside every timed step and the RMSE read back.  P and the SGD
kernel's tile are autotuned, untimed, before the timed steps unless --P is
given.

--impl reference times the FP64 CPU oracle (the only reference there is: the
paper ships no code) on a bounded sample of the same workload.
Multi-GPU: replicas only (one independent job per rank), weak scaling.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Hardware work queues for concurrent streams and graph branches (read when CUDA initialises; the
# default 8 caps the batched-training graph at about 8 concurrent instances).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid")
    ap.add_argument("--P", type=int, default=0, help="strata (0 = workload default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the top-N and online-update measurements")
    ap.add_argument("--no-large", action="store_true", help="skip the full-size Yahoo!-shaped workload")
    ap.add_argument("--epochs", type=int, default=0, help="epochs per job (0 = the workload's; other values are for profiling only)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
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
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_entry(kernel, workload, src_hash):
    """Per-launch DRAM bytes of a kernel on a workload from the committed ncu summary
    (profiles/dram_traffic.json), if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel, {}).get(workload)
        if e and e.get("kernel_source_sha1") == src_hash:
            return e
    except Exception:
        pass
    return None


def kernel_hash(files=("sgd.cu", "common.cuh")):
    h = hashlib.sha1()
    for fn in files:
        with open(os.path.join(ROOT, "paper_2111_11682_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def sgd_bytes_per_epoch(stats, w):
    """Algorithmic bytes of one epoch in the paper's memory model (Sec. 4.2, Alg. 3:
    item parameters stay on chip, u_i and b_i are read and written per rating):
    per rating 4 (user slot) + 1 (rating) + K/8 (mask) + 8F (u_i r/w) + 8 (b_i r/w),
    plus one byte per explicit neighbour rating."""
    nnz = stats["nnz"]
    return nnz * (4 + 1 + w.K / 8 + 8 * w.F + 8) + stats["explicit_neighbours"]


def sgd_min_bytes_per_epoch(stats, w):
    """Compulsory bytes of one epoch: the rating stream (4 + 1 + K/8 B per rating plus the explicit
    neighbour ratings) and one read and one write of every parameter (U, V, b, bhat, W, C, FP32)."""
    params = 4 * (w.M * w.F + w.N * w.F + w.M + w.N + 2 * w.N * w.K)
    return stats["nnz"] * (4 + 1 + w.K / 8) + stats["explicit_neighbours"] + 2 * params


def sig_bytes(w, nnz):
    """Algorithmic bytes of the signature stage (Sec. 4.1, Eq. 3) for one call: the CSC read once
    (4 B row + 1 B rating per rating, 8 B column pointer per item), the users' hash words read once
    (8 W B per user, W = ceil(L bits / 64)), the keys written (4 L B per item) and the kept pre-sign
    sums written (8 B per padded hash bit per item: 64 Wp bits, Wp = W rounded up to 1-4, 8 or 16)."""
    Wh = (w.L * w.bits + 63) // 64
    Wp = Wh if Wh <= 4 else (8 if Wh <= 8 else 16)
    return 5 * nnz + 8 * (w.N + 1) + 8 * Wh * w.M + 4 * w.L * w.N + 8 * 64 * Wp * w.N


# Integer-add peak of the GB300 (nominal): 152 SMs x 128 INT32-capable lanes x 2.07 GHz, in Tops/s
INT32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def measure_signatures(m, col_ptr, row, rc, H, w, reps=10):
    """lshmf_signatures (the Eq. (3) stage alone) on the workload's CSC: CUDA events around one call
    on the current stream, median of `reps` after two warm-ups; roofline of its algorithmic bytes."""
    import torch

    sig = torch.empty((w.L, w.N), dtype=torch.int32, device=row.device)
    ms = []
    stream = torch.cuda.current_stream()
    for k in range(reps + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.signatures(col_ptr, row, rc, H, sig_out=sig)
        b.record(stream)
        b.synchronize()
        if k >= 2:
            ms.append(a.elapsed_time(b))
    m.check()
    med = float(np.median(ms))
    nnz = int(row.numel())
    byts = sig_bytes(w, nnz)
    peak, peak_kind = peaks()
    ach = byts / (med / 1e3) / 1e9
    prof = profile_entry("signatures", w.name, kernel_hash(("simlsh.cu", "common.cuh")))
    # the stage is bound by integer work: Eq. 3 as defined adds +-Psi(r) into L x bits sums per rating
    ops = float(nnz) * w.L * w.bits
    ops_ach = ops / (med / 1e3) / 1e12
    return {"what": "lshmf_signatures: simLSH keys of all items (Eq. 3) and the kept pre-sign sums",
            "ms_median": round(med, 4), "ms_all": [round(x, 4) for x in ms],
            "ratings_per_s": nnz / (med / 1e3),
            "roofline": {"bound": "alu", "achieved": round(ops_ach, 3), "peak": INT32_PEAK_TOPS, "unit": "Tops/s",
                         "frac": round(ops_ach / INT32_PEAK_TOPS, 4),
                         "note": "Eq. 3's signed adds as defined (L x bits per rating) per second, against 152 SMs x "
                                 "128 INT32 lanes x 2.07 GHz (nominal)",
                         "int_adds_per_rating": w.L * w.bits,
                         "hbm_view": {"achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                                      "traffic": prof.get("dram_bytes_per_launch") if prof else None,
                                      "algorithmic_bytes": int(byts), "note": f"frac of {peak_kind} HBM copy bandwidth"}}}


def gpu_job_rmse(ws, d, dev, P=None):
    """The whole job on the GPU through the library (COO -> CSC, neighbour build, layout, every epoch)
    on workload `ws` and its held-out RMSE (Eq. 6)."""
    import torch

    from paper_2111_11682_gb300 import LshMF, Params, config_from_workload

    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    m = LshMF(config_from_workload(ws, P))
    ti, tj, tr = t(d["train_i"], torch.int32), t(d["train_j"], torch.int32), t(d["train_r"], torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(ti, tj, tr)
    nbr = m.build_neighbours(col_ptr, row, rc, t(d["H"].view(np.int64), torch.int64))
    p = Params.from_init(d["U0"], d["V0"], ws.K, dev)
    p.mu = m.prepare_training(ti, tj, tr, nbr)
    for e in range(ws.epochs):
        m.train_epoch(p, e)
    rm = m.rmse(p, t(d["test_i"], torch.int32), t(d["test_j"], torch.int32), t(d["test_r"], torch.uint8))
    m.close()
    return rm


def rmse_parity(gpu, orc, sample, bar=2e-3):
    rel = abs(gpu - orc) / orc
    return {"gpu": gpu, "oracle": orc, "rel": rel, "bar": bar, "pass": bool(rel <= bar), "sample": sample}


def host_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def measure_topn(m, p, w, dev, sizes=(1, 64, 1024, 4096), reps=20, n=10, seed=0):
    """Top-N serving (lshmf_topn, Eq. (1) over all items): latency of one call for batches of
    query users of several sizes (users drawn uniformly, inputs resident in HBM), for the FP32
    path (mode 0) and the BF16 tensor-core candidates + FP32 rerank path (mode 1), and the
    recall@n of mode 1 against mode 0 on the largest batch."""
    import torch

    rng = np.random.default_rng(seed)
    out = {"what": "lshmf_topn: Eq. (1) over all unrated items, top-%d" % n, "modes": {}}
    for mode, name in ((0, "fp32"), (1, "bf16_tc_candidates+fp32_rerank")):
        rows = []
        for bs in sizes:
            users = torch.from_numpy(rng.integers(0, w.M, (reps + 2, bs)).astype(np.int32)).to(dev)
            ms = []
            for r in range(reps + 2):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                m.topn(p, users[r], n, mode=mode)
                b.record()
                torch.cuda.synchronize()
                if r >= 2:
                    ms.append(a.elapsed_time(b))
            ms = np.array(ms)
            rows.append({"users": bs, "p50_ms": round(float(np.percentile(ms, 50)), 4),
                         "p99_ms": round(float(np.percentile(ms, 99)), 4),
                         "items_scored_per_s": bs * w.N / (float(np.median(ms)) / 1e3)})
        out["modes"][name] = rows
    m.check()
    users = torch.from_numpy(rng.integers(0, w.M, sizes[-1]).astype(np.int32)).to(dev)
    i0, _ = m.topn(p, users, n, mode=0)
    i1, _ = m.topn(p, users, n, mode=1)
    i0, i1 = i0.cpu().numpy(), i1.cpu().numpy()
    hits = sum(len(set(a.tolist()) & set(b.tolist())) for a, b in zip(i0, i1))
    out["recall_at_%d_mode1_vs_mode0" % n] = hits / float(n * len(i0))
    return out


def measure_ingest(w, d, P, dev, reps=3, frac=0.01, local_epochs=1):
    """Online update (lshmf_ingest, Sec. 4.3 / Alg. 4) on the workload: the last `frac` of
    users and of items are new; the increment is every rating with a new user or a new item.
    Each repetition rebuilds the model before the update (untimed) and times the ingest call
    with CUDA events (inputs resident in HBM)."""
    import dataclasses

    import torch

    from paper_2111_11682_gb300 import LshMF, Params, config_from_workload

    M_new, N_new = max(1, int(w.M * frac)), max(1, int(w.N * frac))
    M_old, N_old = w.M - M_new, w.N - N_new
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    old = (i < M_old) & (j < N_old)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    oi, oj, orr = t(i[old], torch.int32), t(j[old], torch.int32), t(r[old], torch.uint8)
    ni, nj, nr = t(i[~old], torch.int32), t(j[~old], torch.int32), t(r[~old], torch.uint8)
    H = t(d["H"].view(np.int64), torch.int64)
    Hold = H[:M_old].contiguous()
    times = []
    for rep in range(reps + 1):
        m = LshMF(config_from_workload(dataclasses.replace(w, M=M_old, N=N_old), P))
        col_ptr, row, rc = m.csc_from_coo(oi, oj, orr)
        nbr = torch.zeros((w.N, w.K), dtype=torch.int32, device=dev)
        m.build_neighbours(col_ptr, row, rc, Hold, nbr_out=nbr[:N_old])
        mu = m.prepare_training(oi, oj, orr, nbr[:N_old].contiguous())
        p = Params.from_init(d["U0"], d["V0"], w.K, dev)
        p.mu = mu
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        m.ingest(M_new, N_new, ni, nj, nr, H, nbr, p, local_epochs=local_epochs)
        b.record()
        torch.cuda.synchronize()
        if rep > 0:   # the first repetition is warm-up
            times.append(a.elapsed_time(b))
        m.close()
        del m, col_ptr, row, rc
    ms = float(np.median(times))
    n = int(ni.numel())
    return {"what": "lshmf_ingest (Sec. 4.3, Alg. 4): sums + keys, top-K of new items, local SGD",
            "new_users": M_new, "new_items": N_new, "ratings": n, "local_epochs": local_epochs,
            "ms_median": round(ms, 3), "ms_all": [round(x, 3) for x in times],
            "ratings_per_s": n / (ms / 1e3)}


def measure_serving(w, d, P, dev, frac_users=0.02, frac_items=0.01, rate=4000.0, horizon=4.0, seed=1,
                    users=(1, 16), loguniform=False):
    """Serving loop (serve.Server) under a Poisson mix on the workload: top-N queries of 1-16 users
    (mode 1, top-10) arrive at `rate` per second for `horizon` seconds, and the last `frac_users` of
    users and `frac_items` of items arrive as online updates of lognormal size (median 20k ratings,
    clipped to 1k-1M) at uniform random times.  Queries are merged into calls (continuous batching,
    up to 4 calls in flight on their own streams) and answered from the last published model while
    updates run on their own thread and stream.  Latency is host wall clock from submission to answer."""
    import dataclasses
    import threading

    import torch

    from paper_2111_11682_gb300 import LshMF, Params, config_from_workload
    from paper_2111_11682_gb300.serve import Server, latency_summary, poisson_times, split_summary

    rng = np.random.default_rng(seed)
    M_new, N_new = int(w.M * frac_users), int(w.N * frac_items)
    M_old, N_old = w.M - M_new, w.N - N_new
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    # increments: new users in id order cut to lognormal rating counts; new items spread alike
    per_user = np.bincount(i[i >= M_old] - M_old, minlength=M_new)
    sizes = []
    while sum(sizes) < per_user.sum():
        sizes.append(int(np.clip(rng.lognormal(np.log(20000.0), 1.5), 1000, 1_000_000)))
    cum_u = np.cumsum(per_user)
    ku = np.searchsorted(np.cumsum(sizes), cum_u, side="left")      # increment of each new user
    nk = int(ku.max()) + 1
    kj_new = (np.arange(N_new) * nk) // max(1, N_new)               # increment of each new item
    kr = np.full(len(i), -1, np.int64)
    nu_mask, nj_mask = i >= M_old, j >= N_old
    kr[nu_mask] = ku[i[nu_mask] - M_old]
    kr[nj_mask] = np.maximum(kr[nj_mask], kj_new[j[nj_mask] - N_old])
    # users of increment k are [Mb[k-1], Mb[k]); items likewise
    Mb = [M_old + int(np.searchsorted(ku, k, side="right")) for k in range(nk)]
    Nb = [N_old + int(np.searchsorted(kj_new, k, side="right")) for k in range(nk)]
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    old = kr < 0
    oi, oj, orr = t(i[old], torch.int32), t(j[old], torch.int32), t(r[old], torch.uint8)
    H = t(d["H"].view(np.int64), torch.int64)
    m = LshMF(config_from_workload(dataclasses.replace(w, M=M_old, N=N_old), P))
    col_ptr, row, rc = m.csc_from_coo(oi, oj, orr)
    nbr = torch.zeros((w.N, w.K), dtype=torch.int32, device=dev)
    m.build_neighbours(col_ptr, row, rc, H[:M_old].contiguous(), nbr_out=nbr[:N_old])
    mu = m.prepare_training(oi, oj, orr, nbr[:N_old].contiguous())
    p = Params.from_init(d["U0"], d["V0"], w.K, dev)
    p.mu = mu
    del col_ptr, row, rc
    incs = []
    prevM, prevN = M_old, N_old
    for k in range(nk):
        sel = kr == k
        incs.append((Mb[k] - prevM, Nb[k] - prevN, i[sel], j[sel], r[sel]))
        prevM, prevN = Mb[k], Nb[k]
    qt = poisson_times(rate, horizon, rng)
    lo, hi = users
    if loguniform:          # query sizes log-uniform in [lo, hi]
        qsize = lambda: int(np.exp(rng.uniform(np.log(lo), np.log(hi + 1))))
    else:
        qsize = lambda: int(rng.integers(lo, hi + 1))
    qusers = [rng.integers(0, M_old, min(hi, max(lo, qsize()))).astype(np.int32) for _ in qt]
    ut = np.sort(rng.uniform(0.05, horizon, nk))
    events = sorted([(x, 0, q) for q, x in enumerate(qt)] + [(x, 1, k) for k, x in enumerate(ut)])
    srv = Server(m, p, H, nbr, n=10, mode=1, max_users=4096, depth=4)
    # warm-up: a few queries of each size class and nothing else
    for bs in (1, 16, 256):
        srv.submit_topn(rng.integers(0, M_old, bs).astype(np.int32))
    srv.drain()
    torch.cuda.synchronize()
    srv.calls, srv.users_served, srv.max_inflight = {"topn": 0, "ingest": 0}, 0, 0
    qreq, ureq = [], []

    def produce():
        t0 = time.perf_counter()
        for x, kind, idx in events:
            dt = t0 + x - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            if kind == 0:
                qreq.append(srv.submit_topn(qusers[idx]))
            else:
                ureq.append(srv.submit_ingest(*incs[idx]))
        srv.close()

    import gc

    th = threading.Thread(target=produce)
    gc.collect()          # the request backlog and the model's host state leave the collector's view first
    gc.freeze()
    t0 = time.perf_counter()
    th.start()
    srv.serve_forever(freeze_gc=False)
    th.join()
    gc.unfreeze()
    wall = time.perf_counter() - t0
    m.check()
    # queries answered while some update was running (submitted after its start, answered before its end)
    spans = [(u.done - u.latency, u.done) for u in ureq if u.error is None]
    during = sum(1 for q in qreq if q.error is None and any(a < q.arrival and q.done < b for a, b in spans))
    out = {"what": "serve.Server: Poisson top-N queries (%d-%d users%s, mode 1, top-10) + online updates of lognormal "
                   % (lo, hi, ", log-uniform" if loguniform else "") +
                   "size, queries served from the last published model while updates run",
           "rate_per_s": rate, "horizon_s": horizon, "updates": nk,
           "update_ratings": [int(len(x[2])) for x in incs],
           "queries": latency_summary(qreq), "queries_split": split_summary(qreq), "ingest": latency_summary(ureq),
           "queries_answered_during_an_update": int(during),
           "topn_calls": srv.calls["topn"], "max_calls_in_flight": srv.max_inflight,
           "mean_users_per_call": srv.users_served / max(1, srv.calls["topn"]),
           "users_per_s": srv.users_served / wall, "wall_s": round(wall, 3)}
    for q in srv.qm:
        q.close()
    m.close()
    return out


def measure_generators(w, d, P, dev, reps=3):
    """Neighbour build time of each top-K generator the paper compares (Sec. 5.3 time-overhead
    table): simLSH (lshmf_build_neighbours) and Rand, RP_cos, minHash (p = 3 sub-keys per table)
    through lshmf_build_neighbours_variant, on the workload's CSC (built untimed).  CUDA events
    around one call, median of `reps` after one warm-up."""
    import torch

    import synth
    from paper_2111_11682_gb300 import LshMF, config_from_workload, lshmf

    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    m = LshMF(config_from_workload(w, P))
    col_ptr, row, rc = m.csc_from_coo(t(d["train_i"], torch.int32), t(d["train_j"], torch.int32),
                                      t(d["train_r"], torch.uint8))
    H = t(d["H"].view(np.int64), torch.int64)
    A = t(synth.projections_i16(w.M, w.L * w.bits, 41), torch.int16)
    p_mh = 3 if w.bits % 3 == 0 else 1
    R = t(synth.random_u32(w.M, w.L * p_mh, 43).view(np.int32), torch.int32)
    nbr = torch.empty((w.N, w.K), dtype=torch.int32, device=dev)
    calls = {
        "simLSH": lambda: m.build_neighbours(col_ptr, row, rc, H, nbr_out=nbr),
        "Rand": lambda: m.build_neighbours_variant(lshmf.GEN_RAND, seed=5, nbr_out=nbr, device=dev),
        "RP_cos": lambda: m.build_neighbours_variant(lshmf.GEN_RPCOS, col_ptr, row, rc, A, nbr_out=nbr),
        "minHash (p=%d)" % p_mh: lambda: m.build_neighbours_variant(lshmf.GEN_MINHASH, col_ptr, row, rc, R, p=p_mh,
                                                                   nbr_out=nbr),
    }
    out = {"what": "neighbour build per top-K generator (keys + buckets + top-K rows), ms",
           "L": w.L, "bits": w.bits, "K": w.K, "ms_median": {}}
    for name, fn in calls.items():
        ms = []
        for k in range(reps + 1):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if k > 0:
                ms.append(a.elapsed_time(b))
        out["ms_median"][name] = round(float(np.median(ms)), 3)
    m.check()
    m.close()
    return out


def measure_batch(dev, n_inst=256, E=3, seed=7):
    """Many independent models trained together, shaped like the batched multi-instance workload:
    `n_inst` instances whose size follows one log-uniform draw s in [0, 1] each -- users 1k x 50^s,
    items 500 x 40^s, ratings 10k x 500^s (1k x 500 with 10k ratings up to 50k x 20k with 5M) --
    integer ratings 1-5 with Zipf items, F = 32, K = 16, simLSH neighbours (L = 8 tables x 8 bits),
    Eq. (7) with beta = 0.3.  The autotuner picks each instance's P (least SM-time per epoch among
    4..64; the fastest P for instances that would otherwise be the batch's critical path) and the
    SGD kernel's tile (groups per CTA, blocks in flight).
    Times E epochs of every instance (CUDA events around the whole job, parameters reset untimed):
    per-instance lshmf_train_epoch calls from a host loop (one run), against one CUDA graph of the
    whole job (lshmf_batch) with instances on parallel branches, round-robin or longest-first by the
    autotuner's epoch time, and against one launch of the epoch kernel per epoch for all instances
    (lshmf_batch_create_fused), each median of 3 after one warm-up.  sm_time_bound_ms = E x the sum
    over instances of epoch ms x min(P, SMs) / SMs: the least time the SMs allow when each instance's
    epoch holds min(P, SMs) SMs for its own duration (a fused launch is not held to it)."""
    import dataclasses

    import torch

    import synth
    from paper_2111_11682_gb300 import (OPT_SGD_GROUPS, OPT_SGD_SLOTS, Batch, Config, LshMF, Params, autotune_P,
                                        autotune_tile, config_from_workload, plan_batch_P)

    rng = np.random.default_rng(seed)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    models, inits, nnz_all, timings, data, tiles, t0 = [], [], [], [], [], [], time.time()
    for x in range(n_inst):
        sz = rng.uniform(0.0, 1.0)
        M, N, nnz = int(round(1000 * 50 ** sz)), int(round(500 * 40 ** sz)), int(round(10_000 * 500 ** sz))
        w = dataclasses.replace(synth.TINY, name=f"inst{x}", M=M, N=N, nnz=nnz, F=32, K=16, L=8, bits=8,
                                beta=0.3, seed=1000 + x, test_frac=0.0)
        d = synth.generate(w)
        m0 = LshMF(config_from_workload(w))
        ti, tj, tr = t(d["train_i"], torch.int32), t(d["train_j"], torch.int32), t(d["train_r"], torch.uint8)
        col_ptr, row, rc = m0.csc_from_coo(ti, tj, tr)
        nbr = m0.build_neighbours(col_ptr, row, rc, t(d["H"].view(np.int64), torch.int64))
        p0 = Params.from_init(d["U0"], d["V0"], w.K, dev)
        m, mu, tim = autotune_P(m0.cfg, ti, tj, tr, nbr, p0, candidates=(4, 8, 16), reps=1)
        m0.close()
        p0.mu = mu
        tile, _ = autotune_tile(m, p0, tiles=((3, 0), (2, 0), (1, 0)), reps=1)
        tiles.append(tile)
        timings.append(tim)
        data.append((ti, tj, tr, nbr))
        models.append(m)
        inits.append(p0)
        nnz_all.append(len(d["train_i"]))
    # P per instance for the batch: least SM-time, except instances that would be the critical path
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    plan = plan_batch_P(timings, E, sms)
    moved = 0
    for x, P in enumerate(plan):
        if P != models[x].cfg.P:
            c = models[x].cfg
            m = LshMF(Config.make(c.M, c.N, c.F, c.K, c.L, c.bits, c.psi_pow, P, list(c.alpha), c.beta,
                                  list(c.lambda_), c.rating_scale))
            m.prepare_training(*data[x])
            m.set_option(OPT_SGD_GROUPS, tiles[x][0])
            m.set_option(OPT_SGD_SLOTS, tiles[x][1])
            models[x].close()
            models[x] = m
            moved += 1
    costs = [timings[x][plan[x]] for x in range(n_inst)]
    del data
    setup_s = time.time() - t0
    ps = [p.clone() for p in inits]

    def reset():
        for q, p in zip(ps, inits):
            q.copy_(p)
        torch.cuda.synchronize()

    def timed(fn, reps=3):
        ms = []
        for _ in range(reps):
            reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    def eager():
        for e in range(E):
            for m, q in zip(models, ps):
                m.train_epoch(q, e)

    total = float(sum(nnz_all)) * E
    out = {"what": "%d uneven instances x %d epochs: host loop of lshmf_train_epoch vs one CUDA graph "
                   "(lshmf_batch)" % (n_inst, E),
           "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
           "instances": n_inst, "ratings": int(sum(nnz_all)), "epochs": E,
           "P_histogram": {str(k): int(v) for k, v in zip(*np.unique([m.cfg.P for m in models], return_counts=True))},
           "tile_histogram (groups, slots; 0 = the kernel's default)": {
               str(k): int(v) for k, v in zip(*np.unique(["%d,%d" % t for t in tiles], return_counts=True))},
           "moved_to_fastest_P": moved, "setup_s": round(setup_s, 1), "modes": {}}
    out["sm_time_bound_ms"] = round(E * sum(c * min(m.cfg.P, sms) for c, m in zip(costs, models)) / sms, 2)
    ms = timed(eager, reps=1)      # the autotuner already ran every model's kernels
    out["modes"]["per_instance_calls"] = {"ms": round(ms, 2), "rating_updates_per_s": total / (ms / 1e3)}
    ref = [q.clone() for q in ps]
    fill = int(math.ceil(sms / np.mean([min(m.cfg.P, sms) for m in models])))   # branches that fill the SMs
    for nb, cost in ((32, None), (fill, costs), (2 * fill, costs)):
        b = Batch(models, ps, epoch0=0, epochs=E, branches=nb, cost=cost)
        timed(b.run, reps=1)
        ms = timed(b.run)
        b.check()
        same = all(torch.equal(getattr(q, n), getattr(r, n)) for q, r in zip(ps, ref) for n in ("U", "V", "W"))
        name = "graph_%d_branches_%s" % (nb, "round_robin" if cost is None else "longest_first")
        out["modes"][name] = {"ms": round(ms, 2), "rating_updates_per_s": total / (ms / 1e3),
                              "kernels": b.kernels, "equal_to_per_instance": bool(same)}
        b.close()
    # one launch of the epoch kernel per epoch for all instances (lshmf_batch_create_fused)
    b = Batch(models, ps, epoch0=0, epochs=E, fused=True)
    timed(b.run, reps=1)
    ms = timed(b.run)
    b.check()
    same = all(torch.equal(getattr(q, n), getattr(r, n)) for q, r in zip(ps, ref) for n in ("U", "V", "W"))
    out["modes"]["fused_one_epoch_launch_for_all_instances"] = {
        "ms": round(ms, 2), "rating_updates_per_s": total / (ms / 1e3), "kernels": b.kernels,
        "equal_to_per_instance": bool(same)}
    b.close()
    for m in models:
        m.close()
    return out


def epoch_split(epoch_ms, E):
    """Median time of each job's first epoch and of its later epochs (epoch_ms holds E epochs per
    job, jobs back to back); the later ones are None for a one-epoch job."""
    x = np.asarray(epoch_ms, dtype=np.float64).reshape(-1, E)
    first = float(np.median(x[:, 0]))
    rest = float(np.median(x[:, 1:])) if E > 1 else None
    return first, rest


def max_over_ranks(x: float, world: int, device) -> float:
    """Max of a per-rank value over all ranks of the process group (the slowest replica sets the
    job time); the value itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput of `world` independent replicas that each process `units_per_rank`
    units, timed by the slowest rank (`ms` per step)."""
    return world * units_per_rank / (ms / 1e3)


def sgd_roofline(stats, w, epoch_ms, P):
    peak, peak_kind = peaks()
    ep_med = float(np.median(epoch_ms))
    bytes_ep = sgd_bytes_per_epoch(stats, w)
    achieved = bytes_ep / (ep_med / 1e3) / 1e9
    prof = profile_entry("sgd_epoch", w.name, kernel_hash())
    return {"bound": "hbm", "kernel": "SGD epoch kernel", "achieved": round(achieved, 1),
            "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": prof.get("dram_bytes_per_epoch") if prof else None,
            "traffic_per_launch": prof.get("dram_bytes_per_launch") if prof else None,
            "traffic_note": "ncu DRAM bytes per epoch (one launch), like achieved; from profiles/dram_traffic.json",
            "algorithmic_bytes_per_epoch": int(bytes_ep),
            "min_bytes_per_epoch": int(sgd_min_bytes_per_epoch(stats, w)),
            "min_bytes_achieved_gbs": round(sgd_min_bytes_per_epoch(stats, w) / (ep_med / 1e3) / 1e9, 1),
            "epoch_ms_median": round(ep_med, 3), "P": P, "note": f"frac of {peak_kind} HBM copy bandwidth"}


# P and SGD tile candidates the bench's autotuner tries per workload (others: the workload's P only)
P_CANDIDATES = {"mid-480kx17770-100M": (912, 1216, 1824), "large-1Mx625k-250M": (608, 1216, 1824)}
TILE_CANDIDATES = ((3, 2), (3, 3), (3, 4))


def tune_job(w, dv, dev, candidates=None, tiles=TILE_CANDIDATES):
    """Untimed autotuning before the timed jobs: the workload's neighbours once, then autotune_P over
    the candidate P (fastest epoch) and autotune_tile over the SGD kernel's (groups, slots) at that P.
    Returns (P, tile, {"P_ms": {P: epoch ms}, "tile_ms": {tile: epoch ms}})."""
    from paper_2111_11682_gb300 import LshMF, Params, autotune_P, autotune_tile, config_from_workload

    candidates = candidates or P_CANDIDATES.get(w.name, (w.P,))
    m0 = LshMF(config_from_workload(w))
    col_ptr, row, rc = m0.csc_from_coo(dv["train_i"], dv["train_j"], dv["train_r"])
    nbr = m0.build_neighbours(col_ptr, row, rc, dv["H"])
    del col_ptr, row, rc
    p0 = Params.from_init(dv["U0"], dv["V0"], w.K, dev)
    m, mu, pt = autotune_P(m0.cfg, dv["train_i"], dv["train_j"], dv["train_r"], nbr, p0, candidates=candidates,
                           objective="latency", reps=1)
    m0.close()
    p0.mu = mu
    tile, tt = autotune_tile(m, p0, tiles=tiles, reps=1)
    P = m.cfg.P
    m.close()
    del nbr, p0
    return P, tile, {"P_ms": {str(k): (None if v is None else round(v, 2)) for k, v in pt.items()},
                     "tile_ms": {"%d,%d" % k: round(v, 2) for k, v in tt.items()}}


class Job:
    """One whole training job through the library on device-resident inputs: COO -> CSC, simLSH
    neighbour build, training layout, every epoch, held-out RMSE."""

    def __init__(self, w, P, dv, dev, epochs, tile=(0, 0)):
        from paper_2111_11682_gb300 import OPT_SGD_GROUPS, OPT_SGD_SLOTS, LshMF, Params, config_from_workload

        self.w, self.P, self.dv, self.E = w, P, dv, epochs
        self.m = LshMF(config_from_workload(w, P))
        self.m.set_option(OPT_SGD_GROUPS, tile[0])
        self.m.set_option(OPT_SGD_SLOTS, tile[1])
        self.init = Params.from_init(dv["U0"], dv["V0"], w.K, dev)
        self.p = self.init.clone()
        self.epoch_events = []

    def run(self, src, record_epochs, stream):
        import torch

        m, p = self.m, self.p
        if src is self.dv:
            p.copy_(self.init)
        col_ptr, row, rc = m.csc_from_coo(src["train_i"], src["train_j"], src["train_r"])
        nbr = m.build_neighbours(col_ptr, row, rc, src["H"])
        p.mu = m.prepare_training(src["train_i"], src["train_j"], src["train_r"], nbr)
        for e in range(self.E):
            if record_epochs:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                m.train_epoch(p, e)
                b.record(stream)
                self.epoch_events.append((a, b))
            else:
                m.train_epoch(p, e)
        return m.rmse(p, src["test_i"], src["test_j"], src["test_r"])


def upload(d, dev, pin=True):
    import torch

    host = {k: torch.from_numpy(np.ascontiguousarray(d[k])) for k in
            ("train_i", "train_j", "train_r", "test_i", "test_j", "test_r", "U0", "V0")}
    host["H"] = torch.from_numpy(np.ascontiguousarray(d["H"]).view(np.int64))
    if pin:
        host = {k: v.pin_memory() for k, v in host.items()}
    return host, {k: v.to(dev) for k, v in host.items()}


def measure_large(dev, steps=2, warmup=1):
    """The Yahoo!-shaped large workload at full size on one GPU (1M users x 625k items, 250M ratings
    0..100, F = 128, K = 32, 32 tables x 16 bits, Psi = r^4 with int64 sums, 5 epochs): whole jobs
    timed with CUDA events (inputs resident in HBM), the signature stage alone, both rooflines, and
    the GPU-vs-oracle RMSE gate on a reduced sample of the same shape (4,000 users x 10,000 items,
    1M ratings, P = 64; the full item count would make the oracle's top-K all-pairs)."""
    import dataclasses

    import torch

    import oracle
    import synth

    w = synth.LARGE
    t0 = time.time()
    d = synth.generate(w)
    gen_s = time.time() - t0
    nnz = len(d["train_i"])
    host, dv = upload(d, dev, pin=False)
    del host
    stream = torch.cuda.current_stream()
    P, tile, tuned = tune_job(w, dv, dev)
    torch.cuda.empty_cache()
    job = Job(w, P, dv, dev, w.epochs, tile)
    jobs_ms = []
    for k in range(warmup + steps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rm = job.run(dv, k >= warmup, stream)
        b.record(stream)
        b.synchronize()
        if k >= warmup:
            jobs_ms.append(a.elapsed_time(b))
    stats = job.m.training_stats()
    epoch_ms = [a.elapsed_time(b) for a, b in job.epoch_events]
    col_ptr, row, rc = job.m.csc_from_coo(dv["train_i"], dv["train_j"], dv["train_r"])
    sig = measure_signatures(job.m, col_ptr, row, rc, dv["H"], w)
    job.m.close()
    del col_ptr, row, rc, dv, job
    torch.cuda.empty_cache()
    ms = float(np.median(jobs_ms))
    # RMSE gate on a reduced sample of the same shape: oracle on every host core, GPU through the library
    ws = dataclasses.replace(synth.scaled(w, 0.004), N=10_000, nnz=1_000_000, P=64,
                             name="large-shape 4kx10k-1M")
    ds = synth.generate(ws)
    prev = oracle.set_threads(os.cpu_count() or 1)
    try:
        rm_o = oracle_job(ws, ds)["rmse_heldout"]
    finally:
        oracle.set_threads(prev)
    rm_g = gpu_job_rmse(ws, ds, dev)
    return {"workload": w.name, "M": w.M, "N": w.N, "nnz_train": nnz, "F": w.F, "K": w.K, "L": w.L,
            "bits": w.bits, "psi_pow": w.psi_pow, "epochs": w.epochs, "P": P, "sgd_tile": list(tile),
            "autotune": tuned,
            "value": w.epochs * nnz / (ms / 1e3), "unit": "rating-updates/s", "ms_per_job": round(ms, 2),
            "jobs_ms": [round(x, 2) for x in jobs_ms], "rmse_heldout": rm,
            "epoch_rating_updates_per_s": nnz / (float(np.median(epoch_ms)) / 1e3),
            "epoch_ms_first_and_later": [None if v is None else round(v, 3) for v in epoch_split(epoch_ms, w.epochs)],
            "roofline": {"sgd": sgd_roofline(stats, w, epoch_ms, P), "signatures": sig["roofline"]},
            "signatures": {k: v for k, v in sig.items() if k != "roofline"},
            "rmse_parity": rmse_parity(rm_g, rm_o, ws.name), "layout": stats, "generate_s": round(gen_s, 1)}


def run_ours(args, rank, world, local_rank):
    import torch

    import synth
    from paper_2111_11682_gb300 import launch_count

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = synth.WORKLOADS[args.workload]
    P = args.P or w.P
    t0 = time.time()
    d = synth.generate(w)
    gen_s = time.time() - t0
    E = args.epochs or w.epochs
    nnz = len(d["train_i"])
    host, dv = upload(d, dev)
    stream = torch.cuda.current_stream()
    tile, tuned = (0, 0), None
    if not args.P:            # P and the SGD tile autotuned (untimed) unless P is given
        P, tile, tuned = tune_job(w, dv, dev)
        torch.cuda.empty_cache()
        if world > 1:         # every replica takes rank 0's choice
            import torch.distributed as dist
            ch = torch.tensor([P, tile[0], tile[1]], dtype=torch.int64, device=dev)
            dist.broadcast(ch, 0)
            P, tile = int(ch[0]), (int(ch[1]), int(ch[2]))
    job = Job(w, P, dv, dev, E, tile)
    m, p = job.m, job.p

    # device buffers the end-to-end steps copy their inputs into (allocated once, so that no step
    # waits on the allocator)
    landing = {k: torch.empty(v.shape, dtype=v.dtype, device=dev) for k, v in host.items()} if not args.no_e2e else {}

    def job_e2e():
        src = landing
        for k, v in host.items():
            src[k].copy_(v, non_blocking=True)
        p.U.copy_(src["U0"], non_blocking=True)
        p.V.copy_(src["V0"], non_blocking=True)
        for x in (p.b, p.bh, p.W, p.C):
            x.zero_()
        return job.run(src, False, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        rmse = job.run(dv, False, stream)
    stats = m.training_stats()
    clk = Clocks(local_rank)
    barrier()
    clk.start()
    l0 = launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        rmse = job.run(dv, True, stream)
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    launches = launch_count() - l0
    ms_total = ev0.elapsed_time(ev1)
    epoch_ms = [a.elapsed_time(b) for a, b in job.epoch_events]
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = replica_throughput(E * nnz, world, ms_step)

    e2e = None
    if not args.no_e2e:
        job_e2e()
        clk_e2e = Clocks(local_rank)
        barrier()
        clk_e2e.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            rmse_e2e = job_e2e()
        e1.record(stream)
        barrier()
        clocks_e2e = clk_e2e.stop()
        ms_e2e = e0.elapsed_time(e1) / args.steps
        ms_e2e = max_over_ranks(ms_e2e, world, dev)
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        e2e = {"value": replica_throughput(E * nnz, world, ms_e2e), "unit": "rating-updates/s", "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8, "clocks": clocks_e2e}

    signatures = topn = None
    if rank == 0:
        col_ptr, row, rc = m.csc_from_coo(dv["train_i"], dv["train_j"], dv["train_r"])
        signatures = measure_signatures(m, col_ptr, row, rc, dv["H"], w)
        del col_ptr, row, rc
    if rank == 0 and not args.no_serving:
        topn = measure_topn(m, p, w, dev)
    ingest = serving = serving_uneven = generators = batch = large = None
    if rank == 0 and not args.no_serving:
        m.close()
        ingest = measure_ingest(w, d, P, dev)
        serving = measure_serving(w, d, P, dev)
        serving_uneven = measure_serving(w, d, P, dev, rate=800.0, users=(1, 4096), loguniform=True, seed=2)
        generators = measure_generators(w, d, P, dev)
        batch = measure_batch(dev)
    m.close()
    del job, dv, host
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_large and args.workload != "large":
        large = measure_large(dev)

    roof = sgd_roofline(stats, w, epoch_ms, P)
    out = {"metric": "SGD rating-updates/s per epoch at RMSE parity (whole training job)", "value": value,
           "unit": "rating-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (SGD), int32/int64 (simLSH)", "data": "synthetic (seeded generator, %s)" % w.name,
           "config": {"workload": w.name, "M": w.M, "N": w.N, "nnz_train": nnz, "F": w.F, "K": w.K, "L": w.L,
                      "bits": w.bits, "psi_pow": w.psi_pow, "epochs": E, "P": P, "sgd_tile": list(tile),
                      "autotune": tuned,
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "inputs > L2 (ratings ~%.0f MB)" % (nnz * 9 / 1e6)},
           "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
           "rmse_heldout": rmse, "epoch_rating_updates_per_s": nnz / (float(np.median(epoch_ms)) / 1e3),
           "epoch_ms_first_and_later": [None if v is None else round(v, 3) for v in epoch_split(epoch_ms, E)],
           "layout": stats, "signatures": signatures,
           "topn": topn, "ingest": ingest, "serving": serving,
           "serving_uneven_queries": serving_uneven, "generators": generators, "batch": batch,
           "large": large, "generate_s": round(gen_s, 1)}
    if rank == 0 and not args.no_cpu:
        ws = synth.scaled(w, 0.005)
        ds = synth.generate(ws)
        cb = cpu_baseline(ws, ds)
        out["cpu_baseline"] = cb
        out["rmse_parity"] = rmse_parity(gpu_job_rmse(ws, ds, dev, P), cb["rmse_heldout"], cb["sample"])
        if not out["rmse_parity"]["pass"]:
            out["parity_note"] = "RMSE parity FAILED on the sample: the value is not at RMSE parity"
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def oracle_job(ws, d):
    """The FP64 oracle's whole job on workload `ws`: CSC, signatures, top-K, every epoch, held-out RMSE."""
    import oracle

    t0 = time.time()
    col_ptr, row, r = oracle.csc(ws.M, ws.N, d["train_i"], d["train_j"], d["train_r"])
    sig = oracle.signatures(ws.M, ws.N, ws.L, ws.bits, ws.psi_pow, col_ptr, row, r, d["H"])
    nbr = oracle.topk_buckets(sig, ws.K)
    t_nb = time.time() - t0
    cfg = oracle.cfg_from_workload(ws)
    mu = oracle.mean(d["train_r"], ws.rating_scale)
    po = oracle.Params.init(d["U0"], d["V0"], ws.K)
    t1 = time.time()
    for e in range(ws.epochs):
        oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu, po, e)
    t_ep = (time.time() - t1) / ws.epochs
    rm = oracle.rmse(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu, po, d["test_i"], d["test_j"], d["test_r"])
    total = time.time() - t0
    nnz = len(d["train_i"])
    return {"value": ws.epochs * nnz / total, "total_s": total, "epoch_rating_updates_per_s": nnz / t_ep,
            "neighbour_build_s": round(t_nb, 2), "rmse_heldout": rm, "U": po.U}


def cpu_baseline(ws, d, serial_leg=True):
    """The FP64 oracle as it stands on a bounded sample `ws` of the workload (same N, F, K, L, bits and
    epochs; users and ratings scaled down), whole job, in two legs: one host thread, and every host
    core (OpenMP over the items of Eq. (3) and the blocks of a stratum; bit-identical results)."""
    import oracle

    info = host_info()
    nproc = info["nproc"] or 1
    prev = oracle.set_threads(1)
    try:
        serial = oracle_job(ws, d) if serial_leg else None
        oracle.set_threads(nproc)
        multi = oracle_job(ws, d)
    finally:
        oracle.set_threads(prev)
    if serial is None:
        multi.pop("U")
        nnz = len(d["train_i"])
        return {"value": multi["value"], "unit": "rating-updates/s", "cores": nproc, "kind": "oracle",
                "sample": f"{ws.name}: {ws.M} users x {ws.N} items, {nnz} training ratings, whole job "
                          f"({ws.epochs} epochs) in {multi['total_s']:.1f} s on {nproc} cores",
                "cpu_model": info["cpu_model"], "nproc": nproc,
                "epoch_rating_updates_per_s": multi["epoch_rating_updates_per_s"],
                "neighbour_build_s": multi["neighbour_build_s"], "rmse_heldout": multi["rmse_heldout"]}
    same = bool(np.array_equal(serial.pop("U"), multi.pop("U")))
    nnz = len(d["train_i"])
    sample = (f"{ws.name}: {ws.M} users x {ws.N} items, {nnz} training ratings, whole job ({ws.epochs} epochs) "
              f"in {serial['total_s']:.1f} s on 1 core, {multi['total_s']:.1f} s on {nproc}")
    return {"value": multi["value"], "unit": "rating-updates/s", "cores": nproc, "kind": "oracle", "sample": sample,
            "cpu_model": info["cpu_model"], "nproc": nproc,
            "epoch_rating_updates_per_s": multi["epoch_rating_updates_per_s"],
            "neighbour_build_s": multi["neighbour_build_s"], "rmse_heldout": multi["rmse_heldout"],
            "serial": {"value": serial["value"], "cores": 1,
                       "epoch_rating_updates_per_s": serial["epoch_rating_updates_per_s"],
                       "neighbour_build_s": serial["neighbour_build_s"]},
            "all_core_equals_serial": same}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    w = synth.WORKLOADS[args.workload]
    ws = synth.scaled(w, 0.002)
    ds = synth.generate(ws)
    res = []
    for _ in range(args.warmup):
        cpu_baseline(ws, ds, serial_leg=False)
    t0 = time.time()
    for _ in range(args.steps):
        res.append(cpu_baseline(ws, ds, serial_leg=False))
    total = time.time() - t0
    v = float(np.mean([r["value"] for r in res]))
    cb = dict(res[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": "SGD rating-updates/s per epoch at RMSE parity (whole training job)",
           "value": v, "unit": "rating-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator, %s)" % w.name,
           "config": {"workload": w.name, "sample": cb["sample"]}, "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "rating-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
