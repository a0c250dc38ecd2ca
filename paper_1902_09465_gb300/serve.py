"""Serving loop: k-NN requests against resident datasets, continuously
batched onto the GPU.

A request holds 1..many query rows (pinned host memory), its k and the
dataset it targets. Each resident dataset is served by the engine its
configuration names: the adaptive rounds (the default) or the exact method
(tensor-core screen + FP64 rerank), whichever the autotuner found faster at
the recall target for that dataset. The scheduler keeps a FIFO of arrived requests and a few
in-flight slots, each with its own CUDA stream. Whenever a slot is free it
takes the dataset of the oldest waiting request and packs as many waiting
requests of that dataset as fit the batch limit and the device-memory budget
(the workspace bytes the batch's round state needs) into one mixed launch
(knn_adaptive_ds_multi: every query keeps its own k and its own Philox query
id, so its result is the same alone or in any mix), followed by the FP64
rerank and the copy of the results to pinned host memory. Batches on
different slots overlap on the device; finished slots are retired by polling
their events, which frees their memory for the next admission. Latency is
measured per request from arrival to the moment its results are on the host.

This module is host orchestration only; every step of the k-NN computation
runs in the library's kernels.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import knn


@dataclass
class Request:
    rid: int
    dataset: int
    Q: torch.Tensor          # nq x m float32, pinned host memory
    k: int
    qid: int = 0             # Philox query id of the first query (the others follow)
    t_arrival: float = 0.0
    t_done: float = 0.0
    idx: torch.Tensor | None = None    # nq x k int64 (host), the exact k nearest of each query after rerank
    dist: torch.Tensor | None = None   # nq x k float64 (host)
    batch_size: int = 0                # queries in the launch that served it


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    busy: bool = False
    reqs: list = field(default_factory=list)
    event: torch.cuda.Event | None = None
    bytes: int = 0
    keep: tuple = ()
    hidx: torch.Tensor | None = None
    hdist: torch.Tensor | None = None


@dataclass
class DatasetConfig:
    """Options of the rounds for one resident dataset (from the autotuner)."""
    storage: str = "f32"
    c_alpha: float = 1e-3
    B0: int = 8
    B: int = 8
    grow: int = 1
    threads: int = 512
    bound: str = "exp"
    share: bool = False      # shared coordinates: both Philox masks zero, column-permuted copy
    r0_tensor: bool = False  # with share: round 0 as a tensor-core contraction (knn_opts.r0_tensor)
    replace: bool = True     # False: each pair's draws without replacement (FP32 storage, no sharing)
    method: str = "adaptive"  # or "exact": screen GEMM + select + FP64 rerank (k_max of the batch)


class Server:
    def __init__(self, datasets, configs=None, slots: int = 4, mem_budget: int = 8 << 30, max_batch: int = 1024,
                 delta: float = 0.01, seed: int = 0):
        self.datasets = list(datasets)
        self.configs = list(configs) if configs else [DatasetConfig() for _ in self.datasets]
        self.delta, self.seed = delta, seed
        self.max_batch = max_batch
        self.mem_budget = int(mem_budget)
        self.mem_used = 0
        self.slots = [_Slot(torch.cuda.Stream()) for _ in range(slots)]
        self.queue: list[Request] = []
        self.done: list[Request] = []
        self.launches = 0
        self.peak_mem = 0
        for ds, c in zip(self.datasets, self.configs):
            if c.share and not (getattr(ds, "_shared_seed", None) == seed and c.storage in getattr(ds, "_shared", ())):
                ds.share(seed, copies=(c.storage,))
                ds._shared_seed, ds._shared = seed, (c.storage,)

    # -- request flow
    def submit(self, req: Request):
        """Queues a request. A malformed one is refused here, before it can
        reach a launch that other requests share."""
        if not 0 <= req.dataset < len(self.datasets):
            raise ValueError(f"request {req.rid}: no dataset {req.dataset}")
        ds, cfg = self.datasets[req.dataset], self.configs[req.dataset]
        Q = req.Q
        if not isinstance(Q, torch.Tensor) or Q.dim() != 2 or Q.dtype != torch.float32 or Q.is_cuda:
            raise ValueError(f"request {req.rid}: Q must be a 2-D float32 host tensor")
        if Q.shape[0] < 1 or Q.shape[1] != ds.m:
            raise ValueError(f"request {req.rid}: Q is {tuple(Q.shape)}, the dataset has m = {ds.m}")
        # the adaptive engine returns k + h = 2k candidates per query
        k_cap = min(ds.n, knn.MAX_KH if cfg.method == "exact" else knn.MAX_KH // 2)
        if not 1 <= req.k <= k_cap:
            raise ValueError(f"request {req.rid}: k = {req.k} outside [1, {k_cap}]")
        if req.t_arrival == 0.0:
            req.t_arrival = time.perf_counter()
        self.queue.append(req)

    def _opts(self, d):
        c = self.configs[d]
        o = dict(bound=c.bound, c_alpha=c.c_alpha, B0=c.B0, B=c.B, grow=c.grow, threads=c.threads)
        if c.share:
            o.update(share_points=True, share_queries=True, r0_tensor=c.r0_tensor)
        if not c.replace:
            o["replace"] = False
        return o

    def _state_bytes(self, d, nq, k_max):
        if self.configs[d].method == "exact":
            return self.datasets[d].exact_workspace_size(nq)
        return self.datasets[d].multi_workspace_size(nq, k_max, **self._opts(d))

    def _admit(self, slot: _Slot) -> bool:
        if not self.queue:
            return False
        d = self.queue[0].dataset
        batch, nq, k_max = [], 0, 0
        for r in self.queue:
            if r.dataset != d:
                continue
            if nq + r.Q.shape[0] > self.max_batch and batch:
                break
            kk = max(k_max, r.k)
            need = self._state_bytes(d, nq + r.Q.shape[0], kk)
            if self.mem_used + need > self.mem_budget and batch:
                break
            if self.mem_used + need > self.mem_budget and not batch and self.mem_used > 0:
                return False          # wait for memory to free up
            batch.append(r)
            nq += r.Q.shape[0]
            k_max = kk
        if not batch:
            return False
        for r in batch:
            self.queue.remove(r)
        ds, cfg = self.datasets[d], self.configs[d]
        need = self._state_bytes(d, nq, k_max)
        dev = ds.X.device
        with torch.cuda.stream(slot.stream):
            Qd = torch.empty((nq, ds.m), dtype=torch.float32, device=dev)
            ks = torch.empty(nq, dtype=torch.int32)
            qids = torch.empty(nq, dtype=torch.int64)
            off = 0
            for r in batch:
                c = r.Q.shape[0]
                Qd[off: off + c].copy_(r.Q, non_blocking=True)
                ks[off: off + c] = r.k
                qids[off: off + c] = torch.arange(r.qid, r.qid + c, dtype=torch.int64)
                off += c
            ks_d = ks.to(dev, non_blocking=False)
            qids_d = qids.to(dev, non_blocking=False)
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            if cfg.method == "exact":
                res = None
                ri, rd = ds.exact(Qd, k_max, workspace=ws, stream=slot.stream)
            else:
                res = ds.adaptive_multi(Qd, ks_d, k_max, qids_d, self.delta, self.seed, storage=cfg.storage,
                                        workspace=ws, stream=slot.stream, **self._opts(d))
                ri, rd = knn.rerank(ds.X, Qd, res["idx"], k_max, stream=slot.stream)
            slot.hidx = torch.empty(ri.shape, dtype=torch.int64, pin_memory=True)
            slot.hdist = torch.empty(rd.shape, dtype=torch.float64, pin_memory=True)
            slot.hidx.copy_(ri, non_blocking=True)
            slot.hdist.copy_(rd, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.keep = (Qd, ks_d, qids_d, ws, res, ri, rd)   # alive until the stream is done with them
        slot.busy, slot.reqs, slot.event, slot.bytes = True, batch, ev, need
        self.mem_used += need
        self.peak_mem = max(self.peak_mem, self.mem_used)
        self.launches += 1
        return True

    def _retire(self, slot: _Slot):
        now = time.perf_counter()
        off = 0
        for r in slot.reqs:
            c = r.Q.shape[0]
            r.idx = slot.hidx[off: off + c, : r.k].clone()
            r.dist = slot.hdist[off: off + c, : r.k].clone()
            r.t_done = now
            r.batch_size = slot.hidx.shape[0]
            off += c
            self.done.append(r)
        self.mem_used -= slot.bytes
        slot.busy, slot.reqs, slot.event, slot.bytes, slot.keep = False, [], None, 0, ()

    def poll(self):
        """Retires finished slots and admits waiting requests into free ones."""
        for s in self.slots:
            if s.busy and s.event.query():
                self._retire(s)
        for s in self.slots:
            if not s.busy:
                if not self._admit(s):
                    break

    def busy(self) -> bool:
        return bool(self.queue) or any(s.busy for s in self.slots)

    def drain(self, timeout_s: float = 600.0):
        t_end = time.perf_counter() + timeout_s
        while self.busy():
            self.poll()
            if time.perf_counter() > t_end:
                raise TimeoutError("serving queue did not drain")
            time.sleep(20e-6)

    def run(self, arrivals, timeout_s: float = 600.0):
        """Replays (t_offset_s, Request) arrivals in real time, then drains.
        Returns the finished requests."""
        arrivals = sorted(arrivals, key=lambda a: a[0])
        t0 = time.perf_counter()
        i = 0
        while i < len(arrivals) or self.busy():
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                r = arrivals[i][1]
                r.t_arrival = t0 + arrivals[i][0]
                self.submit(r)
                i += 1
            self.poll()
            if now > timeout_s:
                raise TimeoutError("serving run did not finish")
            time.sleep(20e-6)
        return self.done


def poisson_requests(rate: float, duration: float, pools, max_queries: int = 256, k_range=(1, 100), seed: int = 0):
    """Seeded Poisson arrivals: inter-arrival times ~ Exp(rate) over
    `duration` seconds; each request picks a dataset uniformly, 1..max_queries
    queries (uniform) from that dataset's query pool, and k uniform in k_range.
    Returns [(t_offset, Request)] with pinned host query tensors and disjoint
    Philox query ids."""
    g = np.random.Generator(np.random.PCG64(seed))
    out, t, rid, qid = [], 0.0, 0, 0
    while True:
        t += g.exponential(1.0 / rate)
        if t > duration:
            break
        d = int(g.integers(0, len(pools)))
        nq = int(g.integers(1, max_queries + 1))
        k = int(g.integers(k_range[0], k_range[1] + 1))
        rows = g.integers(0, pools[d].shape[0], size=nq)
        Q = torch.from_numpy(np.ascontiguousarray(pools[d][rows])).pin_memory()
        out.append((t, Request(rid=rid, dataset=d, Q=Q, k=k, qid=qid)))
        rid += 1
        qid += nq
    return out


def latency_stats(done):
    lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in done])
    q = sum(r.Q.shape[0] for r in done)
    t0 = min(r.t_arrival for r in done)
    t1 = max(r.t_done for r in done)
    return {"requests": len(done), "queries": int(q), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "queries_per_s": q / (t1 - t0), "span_s": t1 - t0}
