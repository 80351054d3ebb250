"""BP_LOG: with the variable set, every traced call writes one stderr line with
its host time and every error its status and message; unset, nothing.  Run
in child processes (the setting is read once per process) on calls that need
no GPU: a host-only schedule query and an argument error of bp_create."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
from paper_1010_0012_gb300 import build
lib = ctypes.CDLL(build.build())
out = ctypes.c_void_p()
lib.bp_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
assert lib.bp_create(0, 4, 8, 0, None, ctypes.byref(out)) == 1
rp = (ctypes.c_int32 * 5)(0, 1, 2, 2, 3)
cl = (ctypes.c_int32 * 3)(1, 0, 3)
v = [ctypes.c_int() for _ in range(4)]
assert lib.bp_sparse_schedule(4, rp, cl, 16, *[ctypes.byref(x) for x in v], None, None) == 0
"""


def _run(env_value):
    env = dict(os.environ)
    env.pop("BP_LOG", None)
    if env_value is not None:
        env["BP_LOG"] = env_value
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return [ln for ln in r.stderr.splitlines() if ln.startswith("[bp]")]


def test_log_lines_when_enabled():
    lines = _run("1")
    assert any(ln.startswith("[bp] bp_create ") and ln.endswith("us host") for ln in lines), lines
    assert any(ln.startswith("[bp] error 1: bp_create: W and H") for ln in lines), lines
    assert any(ln.startswith("[bp] bp_sparse_schedule ") for ln in lines), lines


def test_silent_when_unset_or_zero():
    assert _run(None) == []
    assert _run("0") == []
