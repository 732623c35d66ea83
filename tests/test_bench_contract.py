"""The JSON line of bench.py's reference arm (the FP64 oracle on the host cores), CPU only,
with the timed oracle replaced by a stub of known rate: one line from rank 0 with the
contract's keys, a value that is the mean of the steps' rates, ms_per_step = 1000 / value,
cpu_baseline and e2e describing the same run; other ranks print nothing.  Also the summary of
the nvidia-smi clock samples (median and maximum SM clock, throttle reasons seen)."""
import json
from types import SimpleNamespace

import pytest

import bench


def _args(**kw):
    a = dict(steps=3, warmup=2, backend="dino", impl="reference", batch=False)
    a.update(kw)
    return SimpleNamespace(**a)


@pytest.fixture
def stub(monkeypatch):
    calls = []
    walls = iter([1 / 9.0, 1 / 9.0, 1 / 2.0, 1 / 4.0, 1 / 6.0])   # two warm-up steps, then three timed

    class FakePool:
        SAMPLE = bench.OracleDinoPool.SAMPLE

        def __init__(self, *a, **k):
            self.cores = 8

        def step(self, z):
            calls.append(len(z))
            return next(walls), None

        def close(self):
            pass

    monkeypatch.setattr(bench, "OracleDinoPool", FakePool)
    return calls


def test_reference_line(stub, capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_reference(_args())
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert len(stub) == 5 and d["steps"] == 3 and d["warmup"] == 2
    assert d["value"] == pytest.approx(4.0) and d["ms_per_step"] == pytest.approx(250.0)
    assert d["unit"] == d["cpu_baseline"]["unit"] == d["e2e"]["unit"]
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == 8 and "sample" in d["cpu_baseline"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"] and "model" not in d["config"]
    assert d["vs_baseline"] is None and d["dtype"] == "f64"


def test_other_ranks_print_nothing(stub, capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(_args())
    assert capsys.readouterr().out.strip() == "" and stub == []


def test_clock_summary():
    lines = [
        "0, 2070, 2070, 499.88, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1950, 2070, 1390.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2010, 2070, 1200.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",   # unreadable sample
        "garbage\n",
    ]
    c = bench.ClockSampler.summarize(lines)
    assert c["sm_mhz"] == 2010.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.ClockSampler.summarize(["0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active\n"])
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler.summarize([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
