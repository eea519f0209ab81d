"""bench.py's JSON line on CPU: the measurement functions are replaced by fakes
(no GPU here), and the line the driver parses is checked for its keys and
types; the legs that catch device errors are run against a fake solver."""
import argparse
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def bench(monkeypatch):
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench as b
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "Stream", lambda: None)
    monkeypatch.setattr(b, "load_peaks", lambda: (6795.1, "measured"))

    class Clocks:
        def __init__(self, i):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

        def summary(self):
            return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}

    monkeypatch.setattr(b, "ClockSampler", Clocks)
    monkeypatch.setattr(b, "bench_single",
                        lambda *a, **k: (126.0, {"kernel_ms": (0.265, 0.0), "flat_ms": 0.2, "imbalance": 0.0, "newton_nodes": 5,
                                                 "newton_iters": 11, "newton_max_iter": 3}))
    monkeypatch.setattr(b, "bench_e2e", lambda *a, **k: (130.0, 8 * 4096 * 4096, 8 * 4096 * 4096))
    monkeypatch.setattr(b, "oracle_errors",
                        lambda *a, **k: {"melt_2d_fp32": {"max_rel_dtheta": 1e-7, "max_abs_dphi": 1e-6}})
    return b


def test_json_line_keys(bench, capsys):
    args = argparse.Namespace(gpus=1, steps=400, warmup=20, impl="gpu", quick=True, no_cpu=True, n=None,
                              window_step=None, only_bar=False, only_d2q5=False, only_batch=False, only_corner=False,
                              batch_count=256, batch_hi=1024)
    assert bench.run_gpu(args) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["value"] == pytest.approx(4096 * 4096 * 400 / 126.0 / 1e3)
    assert d["ms_per_step"] == pytest.approx(126.0 / 400)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6795.1
    # the flat kernel: two launches of 0.1 ms, each over half of rows 1 .. 4094 outside the W / E groups
    assert r["achieved"] == pytest.approx(72 * (4094 * 4088 / 2) / 0.1e-3 / 1e9)
    assert r["units_per_launch"] == 4094 * 4088 / 2
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert "workload" in d["config"] and d["gpu_launches"] == 6 * 400
    assert d["error_vs_oracle"]["max_rel_dtheta"] == 1e-7
    assert d["newton_mean_iterations_last_step"] == pytest.approx(11 / 5)
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}


class _FakeStefan:
    fail = None

    @classmethod
    def from_case(cls, c, stream=None, **kw):
        return cls()

    def set_method(self, m):
        self.m = m

    def set_ic(self, t):
        pass

    def step(self, n):
        pass

    def sync(self):
        from paper_2505_13097_gb300 import _abi
        if _FakeStefan.fail == self.m:
            raise _abi.LBMError(3, "inner loop at its limit")

    def stats(self):
        return {"newton_max_iter": 7}

    def close(self):
        pass


class _Ev:
    def __init__(self, **k):
        pass

    def record(self, s=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, o):
        return 12.5


@pytest.mark.parametrize("fail", [None, "ILFBM"])
def test_scheme_legs_report_device_errors(bench, fail):
    from paper_2505_13097_gb300 import workloads
    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Event=_Ev, synchronize=lambda: None))
    solver = types.SimpleNamespace(Stefan=_FakeStefan)
    _FakeStefan.fail = fail
    bar = bench.bench_bar_1d(torch, solver, workloads, None, steps=100)
    cav = bench.bench_cavity_d2q9_801(torch, solver, workloads, None, steps=5, warmup_steps=2)
    _FakeStefan.fail = None
    if fail:
        assert "error" in bar["ilfbm"] and "error" in cav["ilfbm"]
        assert "ilfbm_over_irebm" not in bar and "ilfbm_over_irebm" not in cav
    else:
        assert bar["ilfbm_over_irebm"] == pytest.approx(1.0) and cav["irebm_over_eebm"] == pytest.approx(1.0)
