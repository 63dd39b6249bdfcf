"""Pass-by-pass ("re-anchored") comparison of a traced LBG design with the
FP64 oracle -- TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and by the
small-workload report of ``bench.py``; it calls only this package's oracle
functions and numpy).

One near-tie row that a design resolves the other way (legitimately, within
the tolerance) changes every later pass, so two whole designs cannot be
compared once that has happened.  Instead, every pass of the traced design
is checked on its own, from the codebook that pass actually used:

* cell allocation (Sec. 2.2 step 1; Algorithm 1, Cell Allocation): the
  oracle's nearest codevector of every row under that codebook, index for
  index outside near-ties (rows whose two best FP64 distances differ by at
  most ``gap_tol`` relative; there the traced choice must itself be within
  ``gap_tol`` of the minimum);
* distortion (Algorithm 1, IntegrateDistortions): the oracle's D within
  ``d_tol`` relative;
* empty cells: the count of cells no row chose, exact (integer work);
* updation (Sec. 2.2 step 3; Algorithm 1, Updation): after an UPDATE, the next
  pass's codebook against the oracle's centroids of the traced cell table
  (empty cells keep their codevector), within ``c_tol``;
* codebook splitting (Algorithm 1): after a SPLIT, the next stage's first
  codebook against the oracle's split, within ``c_tol``;
* the stop test (Sec. 2.2 step 2, with the readings: D_prev = +inf at every
  stage, the stage ends when D == 0 or (D_prev - D)/D <= theta, or when it has
  run max_passes passes): recomputed from the traced D values it must give the
  traced action exactly; recomputed from the oracle's D values it must agree
  wherever the oracle's ratio is farther from theta than the D tolerance can
  move it;
* after FINISH: the returned codebook, cell table and D are that pass's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import lloyd_step, split, update

UPDATE, SPLIT, FINISH = "update", "split", "finish"


def stop_action(D_prev: float, D: float, theta: float, pass_index: int, max_passes: int,
                n_cur: int, N: int) -> str:
    """Decision after a pass (Sec. 2.2 step 2 with readings R1, R2, R11):
    continue the stage (UPDATE) or end it (SPLIT, or FINISH at N entries)."""
    done = D == 0.0 or (D_prev - D) / D <= theta
    if not done and pass_index + 1 >= max_passes:
        done = True
    if not done:
        return UPDATE
    return FINISH if n_cur >= N else SPLIT


@dataclass
class PassCheck:
    index: int
    stage_n: int
    pass_: int
    action: str
    assign_mismatch: int        # rows whose choice differs from the oracle's (all exempt if ok)
    assign_bad: int             # of those, rows outside the near-tie exemption
    exempt_rows: int            # near-tie rows of the oracle in this pass
    D_rel: float
    empty_ok: bool
    next_rel: float | None      # codebook error of the update / split that follows
    action_ok: bool             # action recomputed from the traced D values
    oracle_action_ok: bool | None   # action recomputed from the oracle's D (None: ambiguous)


@dataclass
class TrajectoryReport:
    passes: list = field(default_factory=list)
    final_ok: bool = False
    notes: list = field(default_factory=list)

    @property
    def worst_D_rel(self) -> float:
        return max((p.D_rel for p in self.passes), default=0.0)

    @property
    def worst_codebook_rel(self) -> float:
        return max((p.next_rel for p in self.passes if p.next_rel is not None), default=0.0)

    @property
    def assign_bad(self) -> int:
        return sum(p.assign_bad for p in self.passes)

    @property
    def exempt_rows(self) -> int:
        return sum(p.exempt_rows for p in self.passes)

    @property
    def assign_exempt_flips(self) -> int:
        return sum(p.assign_mismatch for p in self.passes)

    def summary(self) -> dict:
        return {"passes_checked": len(self.passes),
                "worst_D_rel": self.worst_D_rel,
                "worst_codebook_rel": self.worst_codebook_rel,
                "assign_rows_outside_tolerance": self.assign_bad,
                "near_tie_rows_resolved_otherwise": self.assign_exempt_flips,
                "oracle_near_tie_rows": self.exempt_rows,
                "empty_cell_count_mismatches": sum(not p.empty_ok for p in self.passes),
                "stop_decisions_wrong": sum(not p.action_ok for p in self.passes),
                "stop_decisions_vs_oracle_D_wrong": sum(p.oracle_action_ok is False for p in self.passes),
                "stop_decisions_within_tolerance_band": sum(p.oracle_action_ok is None for p in self.passes),
                "final_state_is_last_pass": self.final_ok}


def compare(X, N: int, delta: float, theta: float, records, pass_C, pass_assign, C_final,
            assign_final, D_final: float, max_passes: int = 1000, gap_tol: float = 1e-5,
            d_tol: float = 1e-5, c_tol: float = 1e-4) -> TrajectoryReport:
    """Check every traced pass of a design (see the module docstring).

    records      per-pass dicts with stage_n, pass, action, D, n_empty
    pass_C       [P, N, L] array: codebook pass p used (first stage_n rows)
    pass_assign  [P, M] array: cell table of pass p
    Returns the per-pass checks; the caller decides what to assert."""
    X = np.ascontiguousarray(X, np.float32)
    Xd = X.astype(np.float64)
    P = len(records)
    if len(pass_C) < P or len(pass_assign) < P:
        raise ValueError("the trace holds fewer passes than the records")
    rep = TrajectoryReport()
    D_prev_gpu = math.inf
    D_prev_ref = math.inf
    for p, r in enumerate(records):
        n = int(r["stage_n"])
        if r["pass"] == 0:
            D_prev_gpu = math.inf
            D_prev_ref = math.inf
        Cp = np.asarray(pass_C[p][:n], np.float64)
        ap = np.asarray(pass_assign[p], np.int32)
        ref = lloyd_step(X, Cp)
        mism = ap != ref.a
        exempt = ref.gap <= gap_tol
        bad = int(np.count_nonzero(mism & ~exempt))
        alt = np.flatnonzero(mism & exempt)
        if alt.size:
            if ap[alt].min() < 0 or ap[alt].max() >= n:
                bad += int(alt.size)
            else:
                d = ((Xd[alt] - Cp[ap[alt]]) ** 2).sum(1)
                bad += int(np.count_nonzero(d > ref.e[alt] * (1 + gap_tol) + 1e-30))
        D = float(r["D"])
        D_rel = abs(D - ref.D) / ref.D if ref.D != 0 else (0.0 if D == 0 else math.inf)
        valid = ap.min() >= 0 and ap.max() < n if ap.size else True
        counts = np.bincount(ap, minlength=n) if valid else np.zeros(n, np.int64)
        empty_ok = bool(valid) and int(np.count_nonzero(counts == 0)) == int(r.get("n_empty", -1))
        want = stop_action(D_prev_gpu, D, theta, int(r["pass"]), max_passes, n, N)
        action_ok = want == r["action"]
        # the oracle's own D values: the same decision unless its ratio lies within the
        # band the D tolerance can move it by
        oracle_ok = None
        if ref.D == 0.0 or D_prev_ref == math.inf:
            oracle_ok = stop_action(D_prev_ref, ref.D, theta, int(r["pass"]), max_passes, n, N) == r["action"]
        else:
            ratio = (D_prev_ref - ref.D) / ref.D
            band = 2.5 * d_tol * max(1.0, D_prev_ref / ref.D)
            if abs(ratio - theta) > band:
                oracle_ok = stop_action(D_prev_ref, ref.D, theta, int(r["pass"]), max_passes, n, N) == r["action"]
        next_rel = None
        if p + 1 < P:
            Cn = np.asarray(pass_C[p + 1], np.float64)
            if r["action"] == UPDATE and valid:
                want_C, _ = update(X, ap, Cp)
                next_rel = _rel(Cn[:n], want_C)
            elif r["action"] == SPLIT:
                next_rel = _rel(Cn[:2 * n], split(Cp, delta))
        rep.passes.append(PassCheck(p, n, int(r["pass"]), r["action"], int(np.count_nonzero(mism)), bad,
                                    int(np.count_nonzero(exempt)), D_rel, empty_ok, next_rel, action_ok,
                                    oracle_ok))
        D_prev_gpu, D_prev_ref = D, ref.D
    if P:
        last = records[-1]
        n = int(last["stage_n"])
        rep.final_ok = (last["action"] == FINISH and n == N
                        and np.array_equal(np.asarray(C_final, np.float32), np.asarray(pass_C[P - 1][:n], np.float32))
                        and np.array_equal(np.asarray(assign_final), np.asarray(pass_assign[P - 1]))
                        and float(D_final) == float(last["D"]))
    return rep


def _rel(C_got, C_want) -> float:
    num = np.abs(np.asarray(C_got, np.float64) - C_want).max(1)
    den = np.maximum(np.abs(C_want).max(1), 1.0)
    return float((num / den).max()) if num.size else 0.0
