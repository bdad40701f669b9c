"""The wait targets of the pipelined Q application (k_apply_q_wave in
csrc/blr_solve.cu), restated as CTA programs and run under random
interleavings on the host.

CTA s applies block s (32 reflectors) of every update QR: step T(i, k, s)
touches rows [32 s, 32 s + 32) of B_k and all of B_i; GEQRT(k)'s reflectors,
applied by CTA 0, touch all of B_k.  A step waits until prog[i] (steps done
on B_i as the lower block) reaches the number of steps on B_i that precede
it in Algorithm 5's order, and until geq[k] (or geq[i] for Q B) is set.
Checked: every program ends (no deadlock), no two steps in flight share a
block row, and each block row sees its steps in the sequential order.  The
same checks must fail for plausible mistakes in the targets.
"""
import random

import pytest


def _sequential(p, q, S, trans):
    ops = []
    if trans:
        for k in range(q):
            ops.append(("G", k))
            ops += [("T", i, k, s) for i in range(k + 1, p) for s in range(S)]
    else:
        for k in range(q - 1, -1, -1):
            ops += [("T", i, k, s) for i in range(p - 1, k, -1) for s in range(S - 1, -1, -1)]
            ops.append(("G", k))
    return ops


def _rows(op, S):
    if op[0] == "G":
        return {(op[1], s) for s in range(S)}
    _, i, k, s = op
    return {(k, s)} | {(i, t) for t in range(S)}


def _programs(p, q, S, trans, target_qt, target_q):
    progs = []
    for s in range(S):
        prog = []
        if trans:
            for k in range(q):
                if s == 0:
                    prog += [("wait", ("prog", k), S * k), ("op", ("G", k)), ("pub", ("geq", k), 1)]
                else:
                    prog.append(("wait", ("geq", k), 1))
                for i in range(k + 1, p):
                    t = target_qt(S, k, s)
                    prog += [("wait", ("prog", i), t), ("op", ("T", i, k, s)), ("pub", ("prog", i), t + 1)]
        else:
            for k in range(q - 1, -1, -1):
                for i in range(p - 1, k, -1):
                    t = target_q(S, i, k, s, q)
                    if i < q:
                        prog.append(("wait", ("geq", i), 1))
                    prog += [("wait", ("prog", i), t), ("op", ("T", i, k, s)), ("pub", ("prog", i), t + 1)]
                if s == 0:
                    prog += [("op", ("G", k)), ("pub", ("geq", k), 1)]
        progs.append(prog)
    return progs


def _kernel_target_qt(S, k, s):
    return S * k + s


def _kernel_target_q(S, i, k, s, q):
    return S * (min(i, q) - 1 - k) + (S - 1 - s)


def _run(p, q, S, trans, seed, target_qt=_kernel_target_qt, target_q=_kernel_target_q):
    rng = random.Random(seed)
    progs = _programs(p, q, S, trans, target_qt, target_q)
    pc, inflight, flags, seen, want = [0] * S, [None] * S, {}, {}, {}
    for op in _sequential(p, q, S, trans):
        for r in _rows(op, S):
            want.setdefault(r, []).append(op)
    while True:
        ready = []
        for c in range(S):
            if inflight[c] is not None:
                ready.append(c)
            elif pc[c] < len(progs[c]):
                ins = progs[c][pc[c]]
                if ins[0] != "wait" or flags.get(ins[1], 0) >= ins[2]:
                    ready.append(c)
        if not ready:
            break
        c = rng.choice(ready)
        if inflight[c] is not None:            # the step ends
            for r in _rows(inflight[c], S):
                seen.setdefault(r, []).append(inflight[c])
            inflight[c] = None
            pc[c] += 1
            continue
        ins = progs[c][pc[c]]
        if ins[0] == "wait":
            pc[c] += 1
        elif ins[0] == "pub":
            flags[ins[1]] = ins[2]
            pc[c] += 1
        else:                                   # the step starts
            for d in range(S):
                if d != c and inflight[d] is not None:
                    assert not (_rows(ins[1], S) & _rows(inflight[d], S)), ("overlap", ins[1], inflight[d])
            inflight[c] = ins[1]
    assert all(pc[c] == len(progs[c]) for c in range(S)), "deadlock"
    assert seen == want, "order"


SHAPES = [(1, 1), (2, 1), (2, 2), (3, 3), (4, 4), (5, 3), (7, 2)]


@pytest.mark.parametrize("trans", [True, False])
def test_wavefront_schedule_is_sequentially_consistent(trans):
    for p, q in SHAPES:
        for S in (1, 2, 3, 4):
            for seed in range(12):
                _run(p, q, S, trans, seed)


@pytest.mark.parametrize("mistake", ["qt_one_early", "q_ignores_q", "q_no_geqrt_wait"])
def test_wavefront_checks_catch_planted_mistakes(mistake):
    """A step admitted one step early, the Q B target that forgets the
    columns past the last diagonal block, or no wait for GEQRT(i) before the
    steps below it: each breaks one of the checks for some interleaving."""
    kw = {}
    if mistake == "qt_one_early":
        kw["target_qt"] = lambda S, k, s: max(0, S * k + s - 1)
        trans = True
    elif mistake == "q_ignores_q":
        kw["target_q"] = lambda S, i, k, s, q: S * (i - 1 - k) + (S - 1 - s)
        trans = False
    else:
        trans = False
    failed = False
    for p, q in SHAPES:
        for S in (2, 3):
            for seed in range(12):
                try:
                    if mistake == "q_no_geqrt_wait":
                        _run_without_geqrt_wait(p, q, S, seed)
                    else:
                        _run(p, q, S, trans, seed, **kw)
                except AssertionError:
                    failed = True
    assert failed


def _run_without_geqrt_wait(p, q, S, seed):
    orig = _programs

    def programs(*a):
        return [[ins for ins in prog if not (ins[0] == "wait" and ins[1][0] == "geq")] for prog in orig(*a)]

    globals()["_programs"] = programs
    try:
        _run(p, q, S, False, seed)
    finally:
        globals()["_programs"] = orig
