"""Makespan model of the tile DAG of Algorithm 4 as the device scheduler runs it.

Host-only analysis, no GPU: given the mean duration of each task type (as
``blr_stats`` reports them: task CTA-seconds / task count), it computes

* the work bound: total task time / number of scheduler CTAs;
* the critical path: the longest chain of dependent tasks (the makespan with
  unlimited CTAs);
* a list schedule: an event simulation of the persistent scheduler with its
  CTA count and its three priority queues (``dag_queue`` in
  ``csrc/blr_dag.h``: GEQRT and TSQRT first, then the updates of the next
  block column, then the rest; first in, first out within a queue).

The DAG is the one of Section 4.3 for the tiled Householder QR of
Algorithm 4, with the edges the scheduler releases (``csrc/blr_dag.h``):

    GEQRT(k)      -> LARFB(k, j) for j > k, TSQRT(k+1, k)
    LARFB(k, j)   -> TPMQRT(k+1, j, k)
    TSQRT(i, k)   -> TSQRT(i+1, k), TPMQRT(i, j, k) for j > k
    TPMQRT(i,j,k) -> TPMQRT(i+1, j, k), and the step-(k+1) task on tile (i, j)

Indices are 0-based (k < q, i in (k, p), j in (k, q)).  A TSQRT releases
its successor TSQRT before it ends: after its first 128-column group, the
successor then running each group once the predecessor has finished it
(update-QR chain pipelining), so the chain advances by about one group's
time per TSQRT.  ``chain`` is the fraction of a TSQRT's time after which
the successor can proceed (1.0: at its end, no pipelining).

Usage: ``python -m paper_2208_06194_gb300.dag_model --p 128 --q 64
--workers 152 --geqrt 15e-3 --larfb 13e-3 --tsqrt 18e-3 --tpmqrt 1.68e-3
--chain 0.67``.
"""
from __future__ import annotations

import argparse
import heapq
import json

GEQRT, LARFB, TSQRT, TPMQRT = 0, 1, 2, 3
NAMES = ("geqrt", "larfb", "tsqrt", "tpmqrt")


def tasks(p: int, q: int):
    """Every task as (type, i, j, k), in the scheduler's id order."""
    for k in range(q):
        yield (GEQRT, k, k, k)
    for k in range(q):
        for j in range(k + 1, q):
            yield (LARFB, k, j, k)
    for k in range(q):
        for i in range(k + 1, p):
            yield (TSQRT, i, k, k)
    for k in range(q):
        for i in range(k + 1, p):
            for j in range(k + 1, q):
                yield (TPMQRT, i, j, k)


def task_counts(p: int, q: int) -> tuple[int, int, int, int]:
    """Tasks per type: q, sum (q-k-1), sum (p-k-1), sum (p-k-1)(q-k-1)."""
    return (q, sum(q - k - 1 for k in range(q)), sum(p - k - 1 for k in range(q)),
            sum((p - k - 1) * (q - k - 1) for k in range(q)))


def successors(p: int, q: int, t):
    ty, i, j, k = t
    out = []
    if ty == GEQRT:
        out += [(LARFB, k, jj, k) for jj in range(k + 1, q)]
        if k + 1 < p:
            out.append((TSQRT, k + 1, k, k))
    elif ty == LARFB:
        if k + 1 < p:
            out.append((TPMQRT, k + 1, j, k))
    elif ty == TSQRT:
        if i + 1 < p:
            out.append((TSQRT, i + 1, k, k))
        out += [(TPMQRT, i, jj, k) for jj in range(k + 1, q)]
    else:
        if i + 1 < p:
            out.append((TPMQRT, i + 1, j, k))
        k1 = k + 1
        if i == k1 and j == k1:
            out.append((GEQRT, k1, k1, k1))
        elif i == k1:
            out.append((LARFB, k1, j, k1))
        elif j == k1:
            out.append((TSQRT, i, k1, k1))
        else:
            out.append((TPMQRT, i, j, k1))
    return out


def indegree(t) -> int:
    ty, _, _, k = t
    prev = 1 if k > 0 else 0
    return (prev, 1 + prev, 1 + prev, 2 + prev)[ty]


def queue(t) -> int:
    ty, _, j, k = t
    if ty in (GEQRT, TSQRT):
        return 0
    return 1 if j == k + 1 else 2


def _is_chain_edge(t, s) -> bool:
    return t[0] == TSQRT and s[0] == TSQRT


def critical_path(p: int, q: int, dur, chain: float = 1.0) -> float:
    """Longest path: earliest finish of the last task with unlimited CTAs.

    dur[type] is the duration of one task of that type (seconds)."""
    start = {}
    pending = {}
    first = (GEQRT, 0, 0, 0)
    start[first] = 0.0
    frontier = [first]
    end = 0.0
    while frontier:
        t = frontier.pop()
        s0 = start[t]
        end = max(end, s0 + dur[t[0]])
        for s in successors(p, q, t):
            ready = s0 + (dur[t[0]] * chain if _is_chain_edge(t, s) else dur[t[0]])
            start[s] = max(start.get(s, 0.0), ready)
            pending[s] = pending.get(s, indegree(s)) - 1
            if pending[s] == 0:
                frontier.append(s)
    return end


def list_schedule(p: int, q: int, dur, workers: int, chain: float = 1.0) -> dict:
    """Event simulation of the persistent scheduler with `workers` CTAs.

    A free CTA takes the oldest task of the highest non-empty queue; a task
    runs for dur[type]; its successors' counters drop when it ends (a
    TSQRT's successor TSQRT after chain * its duration)."""
    ready = [[], [], []]
    seq = 0

    def push(t):
        nonlocal seq
        heapq.heappush(ready[queue(t)], (seq, t))
        seq += 1

    pending = {}

    def drop(s):
        pending[s] = pending.get(s, indegree(s)) - 1
        if pending[s] == 0:
            push(s)

    push((GEQRT, 0, 0, 0))
    total = sum(task_counts(p, q))
    events = []   # (time, order, task, is_early_release)
    now, free, done, busy, ev = 0.0, workers, 0, 0.0, 0
    while done < total:
        while free > 0 and any(ready):
            qi = next(n for n in range(3) if ready[n])
            _, t = heapq.heappop(ready[qi])
            free -= 1
            d = dur[t[0]]
            busy += d
            if t[0] == TSQRT and chain < 1.0:
                heapq.heappush(events, (now + d * chain, ev, t, True))
                ev += 1
            heapq.heappush(events, (now + d, ev, t, False))
            ev += 1
        if not events:
            raise RuntimeError("scheduler model stalled: the DAG has a task that is never released")
        now, _, t, early = heapq.heappop(events)
        if early:
            if t[1] + 1 < p:
                drop((TSQRT, t[1] + 1, t[2], t[3]))
            continue
        free += 1
        done += 1
        for s in successors(p, q, t):
            if not (chain < 1.0 and _is_chain_edge(t, s)):
                drop(s)
    return {"makespan": now, "busy": busy, "utilisation": busy / (workers * now) if now > 0 else 0.0}


def estimate(p: int, q: int, dur, workers: int, chain: float = 1.0) -> dict:
    """Work bound, critical path and list-schedule makespan (seconds)."""
    n = task_counts(p, q)
    work = sum(n[t] * dur[t] for t in range(4))
    ls = list_schedule(p, q, dur, workers, chain)
    return {"workers": workers, "work_bound_s": work / workers,
            "critical_path_s": critical_path(p, q, dur, chain),
            "list_schedule_s": ls["makespan"], "utilisation": ls["utilisation"], "tsqrt_chain": chain}


def durations_from_stats(stats: dict) -> dict:
    """Mean task duration per type from blr_stats (task CTA-seconds / tasks)."""
    return {t: (stats["task_seconds"][t] / stats["tasks"][t]) if stats["tasks"][t] else 0.0 for t in range(4)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--p", type=int, required=True)
    ap.add_argument("--q", type=int, required=True)
    ap.add_argument("--workers", type=int, default=152)
    for name in NAMES:
        ap.add_argument(f"--{name}", type=float, required=True, help=f"seconds per {name.upper()} task")
    ap.add_argument("--chain", type=float, default=1.0,
                    help="fraction of a TSQRT's time after which it releases the next TSQRT")
    a = ap.parse_args(argv)
    dur = {t: getattr(a, NAMES[t]) for t in range(4)}
    print(json.dumps(estimate(a.p, a.q, dur, a.workers, a.chain)))


if __name__ == "__main__":
    main()
