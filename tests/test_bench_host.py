"""The reference arm of bench.py on CPU: the JSON line it prints (one line,
the same metric and unit as the GPU arm, the oracle described as the CPU
baseline, no host-device bytes), alone and as two gloo ranks of a
torch.distributed launch, where rank 0 alone runs and prints and the other
rank exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "water64", "--steps", "1", "--warmup", "0"]


def _env(**kw):
    env = dict(os.environ)
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    env.update({k: str(v) for k, v in kw.items()})
    return env


def _json_lines(text):
    return [json.loads(s) for s in text.splitlines() if s.startswith("{")]


def _check_line(d, n_gpus):
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["n_gpus"] == n_gpus and d["steps"] == 1 and d["warmup"] == 0
    assert d["dtype"] == "f64" and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("water")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, env=_env(),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def test_reference_arm_under_two_ranks_prints_once_from_rank_0():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    procs = [subprocess.Popen([sys.executable, "bench.py", *ARGS], cwd=ROOT,
                              env=_env(RANK=r, LOCAL_RANK=r, WORLD_SIZE=2, MASTER_ADDR="127.0.0.1",
                                       MASTER_PORT=port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in (0, 1)]
    outs = [p.communicate(timeout=600) for p in procs]
    for p, (_, err) in zip(procs, outs):
        assert p.returncode == 0, err[-2000:]
    assert _json_lines(outs[1][0]) == []
    lines = _json_lines(outs[0][0])
    assert len(lines) == 1
    _check_line(lines[0], 2)
