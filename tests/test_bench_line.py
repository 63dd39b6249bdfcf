"""bench.py's GPU arm assembles the JSON line the measurement contract asks for.

The arm needs a GPU, so this test runs it in a child process in which torch's
few CUDA calls and the library's entry points are replaced by stand-ins that
return fixed timings: everything else -- the workload, the oracle's CPU
baseline and the estimate built on it, the roofline and traffic fields, the
e2e leg, the clock record without NVML -- is the bench's own code.  The
numbers are meaningless; the keys, their types and their units are checked.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys, types
import numpy as np
sys.path.insert(0, ROOT)

class FT:
    """A host array standing in for a tensor."""
    def __init__(self, a):
        self.a = np.asarray(a)
    shape = property(lambda self: self.a.shape)
    def cuda(self): return self
    def cpu(self): return self
    def numpy(self): return self.a
    def clone(self): return FT(self.a.copy())
    def pin_memory(self): return self
    def zero_(self): return self

class Event:
    def __init__(self, enable_timing=False): pass
    def record(self, stream=None): pass
    def elapsed_time(self, other): return 0.625

torch = types.ModuleType("torch")
torch.float32, torch.int32 = np.float32, np.int32
torch.from_numpy = FT
torch.empty = lambda shape, dtype=None, device=None: FT(np.zeros(shape, dtype or np.float32))
torch.empty_like = lambda t: FT(np.zeros_like(t.a))
torch.cuda = types.SimpleNamespace(
    is_available=lambda: True, current_device=lambda: 0,
    current_stream=lambda *a: types.SimpleNamespace(cuda_stream=0),
    synchronize=lambda: None, Event=Event,
    nvtx=types.SimpleNamespace(range_push=lambda s: None, range_pop=lambda: None))
sys.modules["torch"] = torch

import bench
import paper_0910_4711_gb300 as lbg
from paper_0910_4711_gb300 import synth

X, N = synth.workload("img2048x8_b8_n4096")
C0 = X[np.random.default_rng(0).choice(X.shape[0], N, replace=False)].copy()

class Train:
    C, D, n_passes = FT(C0), 1.0e9, 111
    @staticmethod
    def passes_per_stage():
        return [2] + [9] * 12 + [1]

lbg.lbg_train = lambda *a, **k: Train
LAUNCHES = [0]
def step(*a, **k):   # each step: ten kernels, as the library would count them
    LAUNCHES[0] += 10
    return types.SimpleNamespace(
        D=1.0e9, n_exact=1248, phase_ms={"prep": 0.023, "assign": 0.506, "exact": 0.048,
                                         "update": 0.072, "total": 0.649})
lbg.lbg_lloyd_step = step
lbg.launch_count = lambda: LAUNCHES[0]
lbg.measure_fp32_peak = lambda stream=None: (80.0, 152)
lbg.step_result_buffer = lambda *a, **k: FT(np.zeros(2))
lbg.read_step_result = lambda buf: (1.0e9, 1248, 0)
if THROTTLE:   # the first timed region reports a thermal slowdown, the next one none
    class Clocks:
        seen = []
        def __init__(self, gpu): pass
        def __enter__(self): return self
        def __exit__(self, *a): pass
        def summary(self):
            Clocks.seen.append(1)
            bad = ["hw_thermal_slowdown"] if len(Clocks.seen) == 1 else []
            return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": bad}
    bench.ClockSampler = Clocks
sys.argv = ["bench.py", "--steps", "2", "--warmup", "3", "--no-grad", "--no-batched",
            "--no-small", "--no-large", "--no-after-split", "--cpu-seconds", "0.2"]
sys.exit(bench.run_ours(bench.parse()))
'''


def _run(throttle):
    env = dict(os.environ, OMP_NUM_THREADS="4")
    code = f"ROOT = {ROOT!r}\nTHROTTLE = {throttle!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_gpu_arm_remeasures_after_a_slowdown():
    line = _run(True)
    assert line["clocks"]["remeasured_after"] == ["hw_thermal_slowdown"]
    assert line["clocks"]["reasons"] == []


def test_gpu_arm_json_line():
    line = _run(False)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "roofline",
                "update_roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["unit"] == "evals/s" and line["n_gpus"] == 1 and line["steps"] == 2
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["dtype"] == "bf16" and line["vs_baseline"] is None
    assert line["value"] == 524288 * 4096 / 0.625e-3
    roof = line["roofline"]
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == roof["achieved"] / roof["peak"]
    assert roof["traffic"] is None or roof["traffic"] > 0
    assert line["update_roofline"]["bound"] == "hbm"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert cb["full_lbg_estimated_s"] > 0 and "estimated" in cb["full_lbg_estimate"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 524288 * 64 * 4 + 4096 * 64 * 4
    assert e2e["d2h_bytes_per_step"] == 4096 * 64 * 4 + 524288 * 4 + 8
    assert line["gpu_launches"] == 20
    assert "reasons" in line["clocks"] and "remeasured_after" not in line["clocks"]
    assert line["other_precision"]["precision"] == "fp32"
    assert line["fp32_peak"] == {"tflops": 80.0, "sms": 152, "how": line["fp32_peak"]["how"]}
    o = line["other_precision"]["roofline"]
    assert o["bound"] == "alu" and o["peak"] == 80.0 and o["frac"] == o["achieved"] / 80.0
    assert line["ms_per_step"] == 0.625 and line["ms_per_step_mean"] == 0.625
