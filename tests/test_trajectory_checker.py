"""The pass-by-pass checker (oracle/trajectory.py) on the CPU: a design traced
by a plain loop over the oracle's own steps passes every check, the checker's
stop rule reproduces the oracle's whole-design trace, and each planted
mistake in a trace (a wrong action, codebook entry, split, cell, distortion or
empty-cell count) is caught."""
import copy

import numpy as np
import pytest

import oracle
from oracle import trajectory as tj
from paper_0910_4711_gb300 import synth


def traced_design(X, N, delta, theta, max_passes=1000):
    """LBG design by a plain loop over oracle steps, every codebook rounded to
    float32 as a float32 design keeps it; returns (records, pass_C, pass_assign,
    C, a, D)."""
    L = X.shape[1]
    C = oracle.mean(X).astype(np.float32)
    recs, pcs, pas = [], [], []
    n = 1
    while True:
        D_prev = np.inf
        for k in range(max_passes):
            ref = oracle.lloyd_step(X, C.astype(np.float64))
            act = tj.stop_action(D_prev, ref.D, theta, k, max_passes, n, N)
            slot = np.zeros((N, L), np.float32)
            slot[:n] = C
            pcs.append(slot)
            pas.append(ref.a.copy())
            recs.append({"stage_n": n, "pass": k, "action": act, "D": ref.D,
                         "n_empty": int(np.count_nonzero(ref.counts == 0))})
            if act != tj.UPDATE:
                break
            C = ref.C.astype(np.float32)
            D_prev = ref.D
        if act == tj.FINISH:
            return recs, np.stack(pcs), np.stack(pas), C, ref.a.copy(), ref.D
        C = oracle.split(C.astype(np.float64), delta).astype(np.float32)
        n *= 2


@pytest.fixture(scope="module")
def design():
    oracle.build()
    X = synth.blocks(synth.make_image(11, 64, 64), 4)    # M = 256, L = 16
    return X, traced_design(X, 8, 0.01, 1e-3)


def run(X, d, **kw):
    recs, pc, pa, C, a, D = d
    return tj.compare(X, 8, 0.01, 1e-3, recs, pc, pa, C, a, D, **kw)


def test_clean_trace_passes_every_check(design):
    X, d = design
    rep = run(X, d)
    s = rep.summary()
    assert s["passes_checked"] == len(d[0]) > 8
    assert s["assign_rows_outside_tolerance"] == 0
    assert s["worst_D_rel"] <= 1e-12
    assert s["worst_codebook_rel"] <= 1e-7         # float32 rounding of the centroids only
    assert s["empty_cell_count_mismatches"] == 0
    assert s["stop_decisions_wrong"] == 0
    assert s["stop_decisions_vs_oracle_D_wrong"] == 0
    assert s["final_state_is_last_pass"]


def test_stop_rule_reproduces_the_oracles_whole_design(design):
    """stop_action applied to the oracle's own per-pass D values gives the
    stage structure of oracle.lbg_train (passes per stage, sizes doubling)."""
    X, _ = design
    o = oracle.lbg_train(X, 8, 0.01, 1e-3)
    n, k, D_prev = o.trace_n.tolist(), o.trace_pass.tolist(), np.inf
    for i in range(len(n)):
        if k[i] == 0:
            D_prev = np.inf
        act = tj.stop_action(D_prev, float(o.trace_D[i]), 1e-3, k[i], 1000, n[i], 8)
        last = i + 1 == len(n)
        want = tj.FINISH if last else (tj.SPLIT if k[i + 1] == 0 else tj.UPDATE)
        assert act == want, (i, act, want)
        D_prev = float(o.trace_D[i])


def test_stop_rule_cases():
    # R2: D == 0 ends a stage; R1: "<=" at the threshold; R11: the pass cap
    assert tj.stop_action(np.inf, 0.0, 1e-3, 0, 1000, 2, 4) == tj.SPLIT
    assert tj.stop_action(np.inf, 5.0, 1e-3, 0, 1000, 2, 4) == tj.UPDATE
    assert tj.stop_action(1.5, 1.0, 0.5, 3, 1000, 4, 4) == tj.FINISH      # ratio 0.5 <= 0.5
    assert tj.stop_action(1.5, 1.0, 0.4999, 3, 1000, 4, 4) == tj.UPDATE
    assert tj.stop_action(2.0, 1.0, 1e-3, 4, 5, 2, 4) == tj.SPLIT          # fifth pass of at most 5


@pytest.mark.parametrize("what", ["action", "codebook", "split", "cell", "D", "empty", "final"])
def test_planted_mistakes_are_caught(design, what):
    X, d = design
    recs, pc, pa, C, a, D = copy.deepcopy(d)
    upd = [i for i, r in enumerate(recs[:-1]) if r["action"] == tj.UPDATE and recs[i + 1]["pass"] > 0]
    spl = [i for i, r in enumerate(recs) if r["action"] == tj.SPLIT]
    if what == "action":
        i = upd[len(upd) // 2]
        recs[i]["action"] = tj.SPLIT
    elif what == "codebook":
        i = upd[-1]
        pc[i + 1][0, 3] += 0.5                      # the update's result, one component
    elif what == "split":
        i = spl[-1]
        n = recs[i]["stage_n"]
        pc[i + 1][[0, 1]] = pc[i + 1][[1, 0]]       # children swapped
    elif what == "cell":
        i = upd[-1]
        n = recs[i]["stage_n"]
        ref = oracle.lloyd_step(X, pc[i][:n].astype(np.float64))
        m = int(np.flatnonzero(ref.gap > 1e-3)[0])
        pa[i][m] = (pa[i][m] + 1) % n               # a clear-cut row moved to another cell
    elif what == "D":
        recs[upd[0]]["D"] *= 1 + 3e-5
    elif what == "empty":
        recs[spl[0]]["n_empty"] += 1
    elif what == "final":
        C = C.copy()
        C[0, 0] += 1.0
    s = tj.compare(X, 8, 0.01, 1e-3, recs, pc, pa, C, a, D).summary()
    caught = (s["stop_decisions_wrong"] or s["worst_codebook_rel"] > 1e-4
              or s["assign_rows_outside_tolerance"] or s["worst_D_rel"] > 1e-5
              or s["empty_cell_count_mismatches"] or not s["final_state_is_last_pass"])
    assert caught, (what, s)
