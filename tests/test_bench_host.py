"""Host logic of the benchmark that needs no GPU: the other workloads' lines that the default line
summarises are taken from child processes, and a child that fails, prints nothing or runs out of
time is recorded as such instead of failing the default line."""
import json
import subprocess

import bench


class _Done:
    def __init__(self, rc, out, err=""):
        self.returncode, self.stdout, self.stderr = rc, out, err


def test_other_configs_summarise_each_child(monkeypatch):
    calls = []

    def fake_run(cmd, capture_output, text, timeout):
        cfg = cmd[cmd.index("--config") + 1]
        calls.append((cfg, cmd, timeout))
        if cfg == "c3":
            line = {"metric": "m", "value": 1.5, "unit": "seeds/s", "ms_per_step": 2.0, "config": {"workload": "w3"},
                    "roofline": {"bound": "alu", "frac": 0.3}, "clocks": {"sm_mhz": 2070.0}, "extra": 1}
            return _Done(0, "build noise\n" + json.dumps(line) + "\n")
        if cfg == "c4":
            return _Done(1, "", "Traceback\nRuntimeError: no GPU\n")
        if cfg == "tri":
            return _Done(0, "nothing that looks like a line\n")
        if cfg == "c5":
            raise subprocess.TimeoutExpired(cmd, timeout)
        return _Done(0, json.dumps({"value": 2.0, "config": {"workload": "wn"}, "passes": {"a": 1}}))

    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    out = bench.other_configs(timeout_s=7)
    assert [c for c, _, _ in calls] == list(bench.OTHER_CONFIGS)
    for cfg, cmd, timeout in calls:
        assert timeout == 7
        assert cmd[cmd.index("--steps") + 1] == "3" and cmd[cmd.index("--warmup") + 1] == "3"
        assert "--no-cpu-baseline" in cmd
    c3 = out["c3"]
    assert c3["workload"] == "w3" and c3["value"] == 1.5 and c3["roofline"]["frac"] == 0.3
    assert "extra" not in c3 and "metric" not in c3
    assert out["c4"]["error"].startswith("exit 1") and "no GPU" in out["c4"]["error"]
    assert out["tri"]["error"].startswith("exit 0")
    assert "timed out" in out["c5"]["error"]
    assert out["next"]["passes"] == {"a": 1}
    assert all("wall_s" in v for v in out.values())
    json.dumps(out)   # the summary goes into the one JSON line
