"""Host logic of the benchmark's optional legs: each runs in a process of its
own, and a leg that crashes, fails or overruns is reported as an error in the
result line instead of ending the measurement.  The child is replaced by small
scripts here, so no GPU is needed."""
from __future__ import annotations

import os
import stat
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _script(tmp_path, body):
    p = tmp_path / "child.sh"
    p.write_text("#!/bin/sh\n" + body + "\n")
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(p)


def test_leg_result_is_the_childs_last_json_line(tmp_path):
    py = _script(tmp_path, 'echo "log line"; echo \'{"a": 1}\'; echo \'{"speedup": 2.5, "args": "\'"$*"\'"}\'')
    out = bench.leg_in_child("batched", ["--steps", "7"], 30, python=py)
    assert out["speedup"] == 2.5
    # the child gets bench.py, the parent's arguments and the leg
    assert out["args"].endswith("bench.py --steps 7 --leg batched")


def test_crashed_leg_is_reported(tmp_path):
    py = _script(tmp_path, 'echo "partial" 1>&2; kill -SEGV $$')
    out = bench.leg_in_child("served", [], 30, python=py)
    assert "error" in out and "-11" in out["error"]
    assert "partial" in out["stderr_tail"]


def test_failed_or_silent_leg_is_reported(tmp_path):
    assert "error" in bench.leg_in_child("served", [], 30, python=_script(tmp_path, "exit 3"))
    assert "error" in bench.leg_in_child("served", [], 30, python=_script(tmp_path, "echo no json"))


def test_overrunning_leg_is_reported(tmp_path):
    out = bench.leg_in_child("served", [], 1.0, python=_script(tmp_path, "exec sleep 20"))
    assert "did not finish" in out["error"]
