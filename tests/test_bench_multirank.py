"""bench.py's multi-rank path on CPU: two `gloo` ranks stand in for two GPUs.

The hot path does not shard (each rank runs an independent replica of the
whole LBG design on its own data), so the only cross-rank steps are the
barrier around the timed region and the max over ranks of the step time; the
job's value is world x per-rank units / that max.  The reference arm runs on
rank 0 only; the other ranks exit at once.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, w, dist = bench.dist_setup(world, backend="gloo")
    assert (r, w) == (rank, world) and dist is not None
    bench.barrier(dist)
    # rank k "measured" a step of (3 + k) ms; every rank must see the slowest one
    ms = bench.max_over_ranks(dist, 3.0 + rank)
    value = bench.job_throughput(w, 1000 * 64, ms / 1e3)
    bench.barrier(dist)

    class Args:
        workload = "img512_b4_n256"
        gpus = world
        steps = 1
        warmup = 0

    ref_rc = bench.run_reference(Args) if rank != 0 else None
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "value": value, "ref_rc": ref_rc}, f)
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == pytest.approx(4.0)            # max over ranks, not the local time
        assert r["value"] == pytest.approx(2 * 64000 / 4e-3)
    assert res[1]["ref_rc"] == 0                        # non-zero ranks skip the reference arm


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    saved = os.environ.pop("RANK", None)
    try:
        assert bench.dist_setup(1) == (0, 1, None)
        assert bench.max_over_ranks(None, 2.5) == 2.5
        assert bench.job_throughput(1, 10, 2.0) == 5.0
    finally:
        if saved is not None:
            os.environ["RANK"] = saved


def test_estimated_full_lbg_time():
    """Stage s of a design (codebook size 2**s) costs passes x M x 2**s evaluations."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.estimated_full_lbg_s([2, 3, 3], 100, 1000.0) == pytest.approx(2.0)
    assert bench.estimated_full_lbg_s([], 100, 1000.0) == 0.0


def test_small_leg_reports_whole_run_comparison():
    """The small leg's comparison with the oracle's whole run, driven here by a
    stand-in for the library (the oracle itself, codebook returned in FP32) so
    that the report code runs without a GPU."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_0910_4711_gb300 import synth

    class T:                       # the few tensor methods small_leg uses
        def __init__(self, a):
            self.a = a

        def cuda(self):
            return self

        def cpu(self):
            return self

        def numpy(self):
            return self.a

    class FakeTorch:
        from_numpy = T

        class cuda:
            @staticmethod
            def synchronize():
                pass

    class FakeLib:
        @staticmethod
        def lbg_train(X, N, delta, theta, precision="fp32", trace=0, trace_passes=0):
            if trace_passes:   # a design traced pass by pass from the oracle's own steps
                from test_trajectory_checker import traced_design
                recs, pc, pa, C, a, D = traced_design(X.a, N, delta, theta)

                class RT:
                    records = [dict(r, ms=0.01) for r in recs]
                    pass_C, pass_assign = T(pc), T(pa)
                RT.C, RT.assign, RT.D = T(C), T(a), D
                return RT
            t = oracle.lbg_train(X.a, N, delta, theta)

            class R:
                C = T(t.C.astype(np.float32))
                D = t.D
                n_passes = len(t.trace_D)

                @staticmethod
                def passes_per_stage():
                    return t.passes_per_stage()
            return R

    class FakeSynth:
        @staticmethod
        def workload(name):
            return synth.blocks(synth.make_image(1, 64, 64), 4), 16

    out = bench.small_leg(FakeLib, FakeSynth, FakeTorch, with_oracle=True)
    assert "vs_oracle_error" not in out, out.get("vs_oracle_error")
    for prec in ("fp32", "bf16"):
        v = out[prec]["vs_oracle"]
        assert v["same_passes_per_stage"] is True
        assert v["D_rel_diff"] == 0.0
        assert v["codebook_max_rel_diff"] < 1e-6
        assert isinstance(v["near_tie_rows_in_oracle_run"], int)
        pp = out[prec]["per_pass_vs_oracle"]
        assert pp["passes_checked"] > 4 and pp["assign_rows_outside_tolerance"] == 0
        assert pp["stop_decisions_wrong"] == 0 and pp["final_state_is_last_pass"]


def test_throttle_rule():
    """Hardware and thermal slowdowns call for a re-measurement; the power cap does not."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.throttled({"reasons": ["hw_thermal_slowdown"]})
    assert bench.throttled({"reasons": ["sw_power_cap", "sw_thermal_slowdown"]})
    assert not bench.throttled({"reasons": ["sw_power_cap"]})
    assert not bench.throttled({"reasons": []})
    assert not bench.throttled({"sm_mhz": None, "reasons": ["no samples"]})
    assert not bench.throttled(None)
