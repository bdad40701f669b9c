"""The makespan model of the scheduler's DAG (host only).

Pins:
* the DAG's edges equal the data dependencies of Algorithm 4 run in program
  order (for each k: GEQRT(k); LARFB(k, j) for j > k; for each i > k,
  TSQRT(i, k) then TPMQRT(i, j, k) for j > k), derived here from what each
  task reads and writes (Sections 3.4.1-3.4.4): read-after-write,
  write-after-write and write-after-read on the tile items;
* the task counts of each type are the closed sums of the loop bounds;
* the critical path is the node-weighted longest path of the same graph
  (networkx), and the list schedule reduces to it with unlimited CTAs and to
  the total work with one CTA.
"""
import itertools

import pytest

from paper_2208_06194_gb300 import dag_model as D


def program_order(p, q):
    for k in range(q):
        yield (D.GEQRT, k, k, k)
        for j in range(k + 1, q):
            yield (D.LARFB, k, j, k)
        for i in range(k + 1, p):
            yield (D.TSQRT, i, k, k)
            for j in range(k + 1, q):
                yield (D.TPMQRT, i, j, k)


def accesses(t):
    """(item, reads, writes) of a task.  A_kk splits into its R (upper) and its
    reflectors Y_kk with T_kk once GEQRT(k) has factored it: TSQRT(i, k)
    updates only R_kk, LARFB(k, j) reads only Y_kk and T_kk."""
    ty, i, j, k = t
    if ty == D.GEQRT:
        return [(("A", k, k), True, True), (("R", k), False, True), (("Y", k), False, True)]
    if ty == D.LARFB:
        return [(("Y", k), True, False), (("A", k, j), True, True)]
    if ty == D.TSQRT:
        return [(("R", k), True, True), (("A", i, k), True, True)]
    return [(("A", i, k), True, False), (("A", k, j), True, True), (("A", i, j), True, True)]


def algorithm4_edges(p, q):
    last_writer, readers, edges = {}, {}, set()
    for t in program_order(p, q):
        for item, r, w in accesses(t):
            if (r or w) and item in last_writer:
                edges.add((last_writer[item], t))
            if w:
                for rd in readers.get(item, ()):
                    if rd != t:
                        edges.add((rd, t))
                last_writer[item] = t
                readers[item] = []
            elif r:
                readers.setdefault(item, []).append(t)
    return edges


def model_edges(p, q):
    return {(t, s) for t in D.tasks(p, q) for s in D.successors(p, q, t)}


SHAPES = [(1, 1), (2, 1), (2, 2), (3, 2), (4, 4), (5, 3), (7, 2), (6, 6), (9, 4)]


@pytest.mark.parametrize("p,q", SHAPES)
def test_edges_are_algorithm4_data_dependencies(p, q):
    assert model_edges(p, q) == algorithm4_edges(p, q)


@pytest.mark.parametrize("p,q", SHAPES)
def test_indegree_counts_predecessors_and_ids_cover_the_dag(p, q):
    ts = list(D.tasks(p, q))
    assert len(ts) == len(set(ts)) == sum(D.task_counts(p, q))
    assert set(ts) == set(program_order(p, q))
    npred = {t: 0 for t in ts}
    for _, s in model_edges(p, q):
        npred[s] += 1
    assert all(npred[t] == D.indegree(t) for t in ts)


def test_task_counts_closed_forms():
    # 65536 x 32768 at b = 512: p = 128, q = 64
    assert D.task_counts(128, 64) == (64, 2016, 6112, 214368)
    for p, q in itertools.product(range(1, 12), range(1, 12)):
        if q > p:
            continue
        g, l, s, t = D.task_counts(p, q)
        assert (g, l) == (q, q * (q - 1) // 2)
        assert s == p * q - q * (q + 1) // 2
        assert t == sum((p - k) * (q - k) for k in range(1, q + 1))
        counts = [0, 0, 0, 0]
        for task in D.tasks(p, q):
            counts[task[0]] += 1
        assert tuple(counts) == (g, l, s, t)


DUR = {D.GEQRT: 5.0, D.LARFB: 3.0, D.TSQRT: 4.0, D.TPMQRT: 1.0}


@pytest.mark.parametrize("p,q", [(3, 2), (5, 3), (6, 6), (9, 4)])
def test_critical_path_is_the_longest_weighted_path(p, q):
    nx = pytest.importorskip("networkx")
    g = nx.DiGraph()
    for t in D.tasks(p, q):
        g.add_node(t)
    # node weights as edge weights into a sink: longest path = max over paths of the sum of durations
    for t, s in model_edges(p, q):
        g.add_edge(t, s, w=DUR[t[0]])
    for t in D.tasks(p, q):
        g.add_edge(t, "end", w=DUR[t[0]])
    want = nx.dag_longest_path_length(g, weight="w")
    assert D.critical_path(p, q, DUR) == pytest.approx(want)


@pytest.mark.parametrize("p,q", [(3, 2), (5, 3), (6, 6), (9, 4)])
@pytest.mark.parametrize("chain", [1.0, 0.5])
def test_list_schedule_limits(p, q, chain):
    n = D.task_counts(p, q)
    work = sum(n[t] * DUR[t] for t in range(4))
    one = D.list_schedule(p, q, DUR, 1, chain)
    assert one["makespan"] == pytest.approx(work) and one["utilisation"] == pytest.approx(1.0)
    wide = D.list_schedule(p, q, DUR, 10 ** 6, chain)
    assert wide["makespan"] == pytest.approx(D.critical_path(p, q, DUR, chain))
    mid = D.list_schedule(p, q, DUR, 3, chain)["makespan"]
    assert max(work / 3, D.critical_path(p, q, DUR, chain)) - 1e-9 <= mid <= work + 1e-9


def test_early_tsqrt_release_shortens_only_the_tsqrt_chain():
    p, q = 9, 4
    full, early = D.critical_path(p, q, DUR, 1.0), D.critical_path(p, q, DUR, 0.5)
    assert early < full
    # with free TSQRTs the chain option changes nothing
    free = dict(DUR)
    free[D.TSQRT] = 0.0
    assert D.critical_path(p, q, free, 0.5) == pytest.approx(D.critical_path(p, q, free, 1.0))


def test_durations_from_stats_and_estimate():
    stats = {"tasks": list(D.task_counts(9, 4)), "task_seconds": [20.0, 18.0, 104.0, 44.0]}
    dur = D.durations_from_stats(stats)
    assert dur == {0: 5.0, 1: 3.0, 2: 4.0, 3: 1.0}
    e = D.estimate(9, 4, dur, 4)
    assert e["work_bound_s"] == pytest.approx(sum(stats["task_seconds"]) / 4)
    assert e["list_schedule_s"] >= max(e["work_bound_s"], e["critical_path_s"]) - 1e-9


@pytest.fixture(scope="module")
def lib():
    import os
    from paper_2208_06194_gb300 import blr
    if not os.path.exists(blr.LIB_PATH):
        from paper_2208_06194_gb300 import build
        build.build()
    return blr


@pytest.mark.parametrize("p,q", SHAPES + [(16, 8), (12, 12)])
def test_scheduler_formulas_release_exactly_algorithm4_dependencies(lib, p, q):
    """The ids, decoding and successor formulas the scheduler kernel runs
    (csrc/blr_dag.h, read through the host-only blr_dag_task) give the same
    graph as Algorithm 4's data dependencies, and number the tasks in the
    model's order."""
    order = list(D.tasks(p, q))
    edges = set()
    for tid, t in enumerate(order):
        task, succ = lib.blr_dag_task(p, q, tid)
        assert task == t, (tid, task, t)
        assert len(succ) == len(set(succ))
        edges |= {(t, order[s]) for s in succ}
    assert edges == algorithm4_edges(p, q)


def test_dag_task_rejects_bad_arguments(lib):
    for args in [(2, 3, 0), (0, 0, 0), (4, 2, -1), (4, 2, sum(D.task_counts(4, 2)))]:
        with pytest.raises(lib.BLRError):
            lib.blr_dag_task(*args)
