"""Continuous-batching request loop for MDFS scans on one GPU.

A ``Server`` owns ``n_slots`` worker threads, each bound to its own CUDA
stream.  The C library keeps one workspace per stream, so a slot's device
buffers stay resident across the jobs it runs; the library grows a buffer when
a job needs more and keeps it afterwards.  The scheduler therefore charges
each slot what it retains, per buffer group: the largest estimate of that
group over the jobs the slot has run since its workspace was last freed.  Jobs
are admitted in arrival order as soon as a slot is free and the retained
bytes of all slots, with the job's groups merged into its slot's, fit the
memory budget.  When they do not, the slot frees its own workspace if that
makes the job fit, and otherwise asks idle slots to free theirs
(``mdfs_release_stream``).  Jobs that arrive while others are on the GPU
join as slots and memory free up, and their work overlaps on the device
(different streams).  A job is one ``mdfs_max_ig`` scan (IG^k_max, Eq. 1 of
arXiv 1811.00631) followed by the chi^2 / extreme-value fit ``mdfs_ig_lim``
(section "Theory").  The scan is deterministic, so a job's result is the same
alone or in a mix.

The scheduler is independent of the GPU: ``Server`` takes an ``executor``
callable, and the default one runs the job through the C ABI on the slot's
stream.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time
from concurrent.futures import Future
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Job:
    x: object                 # (M, N) float32 or int8, host array or CUDA tensor
    y: object                 # (N,) uint8
    k: int = 2
    divisions: int = 1
    discretizations: int = 1
    range_: float = 0.0
    pc_xi: float = 0.25
    seed: int = 0
    alpha: float = 0.05       # level of the IG_lim fit (None: skip the fit)
    tag: object = None
    deadline_s: Optional[float] = None  # latest start, in seconds after submission (None: no deadline)


@dataclasses.dataclass
class Result:
    ig: np.ndarray
    tuples: np.ndarray
    disc: np.ndarray
    p_values: Optional[np.ndarray]
    ig_lim: Optional[float]
    n_eff: Optional[float]
    submit_t: float
    start_t: float
    end_t: float
    slot: int
    tag: object = None

    @property
    def latency(self) -> float:
        return self.end_t - self.submit_t


def job_device_parts(M: int, N: int, k: int, divisions: int, discretizations: int, x_itemsize: int = 4) -> dict:
    """Upper estimate of the device memory one job holds in its slot's
    workspace, per group of library buffers: "inputs" (staged x and y, the
    class order, entropy tables), "planes" (bit planes, single counts, keys),
    "onehot" (the tensor-core operand of k = 2 with c <= 3 and k = 3 with
    c = 2), "k3tc" (the relabelled operand and the pair records of the k = 3
    tensor path), "pairs" (pair tables of the generic k = 3 path) and "tables"
    (pair, triple and quadruple tables of k = 4, 5 with two classes; the work
    items of k = 4, 5 with three or four).  Tables are processed in
    chunks of discretisations that fit a 4 GB budget (at least one
    discretisation per chunk)."""
    c = divisions + 1
    P = c - 1
    D = discretizations
    words = (N + 31) // 32 + 5
    kp = ((N + 127) // 128 + 1) * 128

    def chunked(per_disc: int) -> int:
        nd = max(1, min(D, (4 << 30) // max(per_disc, 1)))
        return nd * per_disc

    parts = {"inputs": M * N * x_itemsize + N * 5 + 3 * (N + 1) * 8 + (1 << 20),
             "planes": D * M * P * words * 4 + D * M * (P * 8 + 8) + M * 8}
    if k == 2 and c <= 3:
        parts["onehot"] = D * M * P * kp
    elif k == 3 and c == 2:
        parts["onehot"] = D * M * kp
        parts["k3tc"] = D * M * kp + D * M * 16 + chunked(M * M * 8)
    elif k == 3:
        parts["pairs"] = chunked(M * M * (8 + P * P * 8))
    elif k in (4, 5) and c != 2:
        parts["tables"] = M * M * 8 + (1 << 20)  # the generic scan keeps only its pair work items
    elif k in (4, 5):
        per_disc = M * M * 16 + math.comb(M, 3) * 12
        if k == 5:
            per_disc += math.comb(M, 4) * 12 + M * 8
        parts["tables"] = chunked(per_disc) + (1 << 21)
    return {g: int(b * 1.15) for g, b in parts.items()}


def job_device_bytes(M: int, N: int, k: int, divisions: int, discretizations: int, x_itemsize: int = 4) -> int:
    """Total of job_device_parts: the device bytes one job needs in an empty slot."""
    return sum(job_device_parts(M, N, k, divisions, discretizations, x_itemsize).values())


def _parts(need) -> dict:
    """An estimate as buffer groups (a plain byte count is one group)."""
    return dict(need) if isinstance(need, dict) else {"all": int(need)}


def _merged(held: dict, need: dict) -> dict:
    return {g: max(held.get(g, 0), need.get(g, 0)) for g in set(held) | set(need)}


class Server:
    """Admits jobs into ``n_slots`` concurrent slots under a device-memory budget."""

    def __init__(self, n_slots: int = 4, memory_budget: Optional[int] = None, device: int = 0,
                 executor: Optional[Callable] = None, estimate: Callable = job_device_parts,
                 log_path: Optional[str] = None, release_workspace: Optional[Callable] = None):
        """estimate(M, N, k, divisions, discretizations, itemsize) gives a job's
        device bytes, as a dict of buffer groups or one number; release_workspace(slot)
        frees a slot's library workspace (default: mdfs_release_stream on the
        slot's stream; with a custom executor and no callback it only resets the
        bookkeeping)."""
        self.n_slots = n_slots
        self._log_path = log_path  # JSON line per finished, failed or expired job
        self._log_lock = threading.Lock()
        self.log_errors = 0
        self.device = device
        self.estimate = estimate
        if memory_budget is None:
            memory_budget = self._default_budget(device) if executor is None else 1 << 40
        self.budget = int(memory_budget)
        self._executor = executor
        self._release_cb = release_workspace
        self._streams = [None] * n_slots
        self._staging = [None] * n_slots  # pinned host buffers per slot (GPU executor)
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._held = [dict() for _ in range(n_slots)]  # bytes retained per buffer group, per slot
        self._busy = [False] * n_slots
        self._shrink = False  # the head job waits for idle slots to free their workspaces
        self.workspace_releases = 0
        self._running = 0
        self._closed = False
        self.expired = 0
        self._n_deadline = 0  # queued jobs that carry a deadline
        self.peak_in_use = 0
        self.peak_running = 0
        self._threads = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(n_slots)]
        for t in self._threads:
            t.start()

    @staticmethod
    def _default_budget(device: int) -> int:
        import torch
        free, _total = torch.cuda.mem_get_info(device)
        return int(free * 0.8)

    # ------------------------------------------------------------------
    def submit(self, job: Job) -> Future:
        fut: Future = Future()
        M, N = int(job.x.shape[0]), int(job.x.shape[1])
        itemsize = 1 if str(getattr(job.x, "dtype", "")).endswith("int8") else 4
        need = _parts(self.estimate(M, N, job.k, job.divisions, job.discretizations, itemsize))
        if sum(need.values()) > self.budget:
            fut.set_exception(MemoryError(f"job needs ~{sum(need.values())} device bytes, budget is {self.budget}"))
            return fut
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            self._purge_expired()
            self._queue.append((job, fut, need, time.perf_counter()))
            self._n_deadline += getattr(job, "deadline_s", None) is not None
            self._cv.notify_all()
        return fut

    def close(self, wait: bool = True):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        if wait:
            for t in self._threads:
                t.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def _purge_expired(self):
        """Drops queued jobs whose start deadline has passed; their futures get
        TimeoutError.  Runs whenever the scheduler looks at the queue (a job
        arrives, a slot asks for work, or an idle slot's timed wait ends).
        Caller holds the lock."""
        if not self._n_deadline:
            return
        now = time.perf_counter()
        keep = collections.deque()
        for item in self._queue:
            job, fut, _need, t_sub = item
            dl = getattr(job, "deadline_s", None)
            if dl is not None and now - t_sub > dl:
                fut.set_exception(TimeoutError(f"job {job.tag!r} not started within its deadline of {dl} s"))
                self._log(job, "expired", t_sub, None, now, None)
                self.expired += 1
                self._n_deadline -= 1
            else:
                keep.append(item)
        self._queue = keep

    def _deadline_wait(self):
        """Seconds until the earliest queued start deadline (None: no deadline)."""
        if not self._n_deadline:
            return None
        now = time.perf_counter()
        waits = [getattr(j, "deadline_s") - (now - t) for j, _f, _n, t in self._queue
                 if getattr(j, "deadline_s", None) is not None]
        return max(1e-3, min(waits)) if waits else None

    @property
    def in_use(self) -> int:
        """Device bytes the slots retain (estimate), running or idle."""
        with self._cv:
            return self._held_total()

    def _held_total(self, skip: int = -1) -> int:
        return sum(sum(h.values()) for s, h in enumerate(self._held) if s != skip)

    def _next(self, slot: int):
        """Head-of-line admission: the oldest job runs as soon as it fits."""
        while True:
            with self._cv:
                while True:
                    self._purge_expired()
                    mine = sum(self._held[slot].values())
                    if self._shrink and mine > 0:
                        break  # idle: free this slot's workspace for the waiting head job
                    if self._queue:
                        job, fut, need, t_sub = self._queue[0]
                        others = self._held_total(skip=slot)
                        merged = _merged(self._held[slot], need)
                        if others + sum(merged.values()) <= self.budget:
                            self._queue.popleft()
                            self._n_deadline -= getattr(job, "deadline_s", None) is not None
                            self._held[slot] = merged
                            self._busy[slot] = True
                            self._shrink = False
                            self._running += 1
                            self.peak_in_use = max(self.peak_in_use, self._held_total())
                            self.peak_running = max(self.peak_running, self._running)
                            return job, fut, need, t_sub
                        if mine > 0 and others + sum(need.values()) <= self.budget:
                            break  # fits once this slot's retained buffers are freed
                        if any(not self._busy[s] and self._held[s] for s in range(self.n_slots) if s != slot):
                            self._shrink = True
                            self._cv.notify_all()
                    elif self._closed:
                        return None
                    self._cv.wait(self._deadline_wait())
            # outside the lock: the slot's workspace is freed before its bytes are
            # returned to the budget
            self._free_workspace(slot)
            with self._cv:
                self._held[slot] = {}
                self.workspace_releases += 1
                self._cv.notify_all()

    def _free_workspace(self, slot: int):
        if self._release_cb is not None:
            self._release_cb(slot)
        elif self._executor is None and self._streams[slot] is not None:
            from . import mdfs
            mdfs.release_stream(self._streams[slot])

    def _release(self, slot: int):
        with self._cv:
            self._busy[slot] = False
            self._running -= 1
            self._cv.notify_all()

    def _worker(self, slot: int):
        ctx = None
        if self._executor is None:
            import torch
            torch.cuda.set_device(self.device)
            ctx = torch.cuda.Stream(self.device)
            self._streams[slot] = ctx
        staging = _Staging()
        self._staging[slot] = staging
        while True:
            item = self._next(slot)
            if item is None:
                return
            job, fut, need, t_sub = item
            t0 = time.perf_counter()
            try:
                if self._executor is not None:
                    out = self._executor(job, slot)
                else:
                    out = _run_on_gpu(job, ctx, self.device, staging)
                t1 = time.perf_counter()
                fut.set_result(Result(*out, submit_t=t_sub, start_t=t0, end_t=t1, slot=slot, tag=job.tag))
                self._log(job, "ok", t_sub, t0, t1, slot)
            except BaseException as e:  # the job failed; the slot keeps serving
                fut.set_exception(e)
                self._log(job, f"error: {type(e).__name__}: {e}", t_sub, t0, time.perf_counter(), slot)
            finally:
                self._release(slot)

    def _log(self, job, status: str, t_sub: float, t_start, t_end: float, slot):
        """Appends one JSON line per job to log_path: shape, work, queue wait,
        run time, latency, evaluation rate and status."""
        if not self._log_path:
            return
        import json
        M, N = int(job.x.shape[0]), int(job.x.shape[1])
        evals = job_evals(M, job.k, job.discretizations) if M >= job.k else 0.0
        run_s = (t_end - t_start) if t_start is not None else None
        rec = {"tag": job.tag if isinstance(job.tag, (int, float, str)) or job.tag is None else str(job.tag),
               "N": N, "M": M, "k": job.k, "classes": job.divisions + 1, "discretizations": job.discretizations,
               "evals": evals, "queue_s": (t_start if t_start is not None else t_end) - t_sub, "run_s": run_s,
               "latency_s": t_end - t_sub, "evals_per_s": evals / run_s if run_s else None, "slot": slot,
               "status": status}
        try:  # a record that cannot be written must not take down the slot
            with self._log_lock, open(self._log_path, "a") as f:
                f.write(json.dumps(rec) + "\n")
        except (OSError, TypeError, ValueError):
            self.log_errors += 1


class _Staging:
    """Page-locked host buffers of one slot.  A host input is copied into the
    input buffer and moved to the device asynchronously on the slot's stream;
    the job's results are packed into one device buffer and come back in one
    device-to-host copy.  A slot runs one job at a time and waits for its
    stream before the next, so the buffers are free again when a job starts."""

    def __init__(self):
        self.h_in = None
        self.h_out = None
        self.h2d_bytes = 0
        self.d2h_bytes = 0

    @staticmethod
    def _grow(buf, nbytes: int):
        import torch
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(int(nbytes * 1.25), 1 << 20), dtype=torch.uint8, pin_memory=True)
        return buf

    def inputs(self, arrays, device: int):
        """Device tensors of the host arrays (CUDA tensors pass through)."""
        import torch
        host = [np.ascontiguousarray(a) for a in arrays if not getattr(a, "is_cuda", False)]
        offs, total = [], 0
        for a in host:
            offs.append(total)
            total += (a.nbytes + 255) & ~255
        if total:
            self.h_in = self._grow(self.h_in, total)
        out, h = [], 0
        for a in arrays:
            if getattr(a, "is_cuda", False):
                out.append(a)
                continue
            a = host[h]
            view = self.h_in[offs[h]:offs[h] + a.nbytes].numpy().view(a.dtype).reshape(a.shape)
            np.copyto(view, a)
            t = self.h_in[offs[h]:offs[h] + a.nbytes].view(torch.from_numpy(a[:0]).dtype).view(a.shape)
            out.append(t.to(f"cuda:{device}", non_blocking=True))
            self.h2d_bytes += a.nbytes
            h += 1
        return out

    def results(self, tensors, stream):
        """numpy copies of the CUDA tensors after one packed read (None stays None)."""
        import torch
        live = [t.contiguous() for t in tensors if t is not None]
        flat = [t.reshape(-1).view(torch.uint8) for t in live]
        sizes = [f.numel() for f in flat]
        total = sum(sizes)
        packed = torch.cat(flat) if len(flat) > 1 else flat[0]
        self.h_out = self._grow(self.h_out, total)
        self.h_out[:total].copy_(packed, non_blocking=True)
        stream.synchronize()
        self.d2h_bytes += total
        host = self.h_out[:total].numpy()
        out, o, i = [], 0, 0
        for t in tensors:
            if t is None:
                out.append(None)
                continue
            n = sizes[i]
            dt = torch.empty(0, dtype=t.dtype).numpy().dtype
            out.append(host[o:o + n].view(dt).reshape(tuple(t.shape)).copy())
            o += n
            i += 1
        return out


def _run_on_gpu(job: Job, stream, device: int, staging: Optional[_Staging] = None):
    import torch

    from . import mdfs
    staging = staging or _Staging()
    with torch.cuda.device(device), torch.cuda.stream(stream):
        y_in = job.y if getattr(job.y, "is_cuda", False) else np.asarray(job.y, dtype=np.uint8)
        x, y = staging.inputs([job.x, y_in], device)
        ig, tu, di = mdfs.max_ig(x, y, job.k, job.divisions, job.discretizations, job.range_, job.pc_xi, job.seed)
        p_t = lim = neff = None
        if job.alpha is not None:
            try:
                p_t, lim, neff = mdfs.ig_lim(ig, job.k, job.divisions, job.discretizations, None, job.alpha)
            except mdfs.MdfsError as e:
                if e.code != -2:  # no variable with IG > 0: no fit for this job
                    raise
        ig_h, tu_h, di_h, p = staging.results([ig, tu, di, p_t], stream)
        return ig_h, tu_h, di_h, p, lim, neff


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "n": int(len(lat))}


def job_evals(M: int, k: int, discretizations: int) -> float:
    """Unordered k-tuple x discretisation evaluations of one job."""
    return float(math.comb(M, k)) * discretizations
