"""The reference arm of bench.py times the FP64 oracle only: it must not load
or call the CUDA library, not even for an input such as the time step."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import io, contextlib, runpy, sys
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
            "--ref-seconds", "0.5"]
buf = io.StringIO()
with contextlib.redirect_stdout(buf):
    runpy.run_path("bench.py", run_name="__main__")
maps = open("/proc/self/maps").read()
print(buf.getvalue().strip().splitlines()[-1])
print("LIBFDWAVE" if "libfdwave" in maps else "NO_LIBFDWAVE")
print("FDWAVE_MODULE" if "paper_1609_03361_gb300.fdwave" in sys.modules else "NO_FDWAVE_MODULE")
"""


def test_reference_arm_loads_only_the_oracle():
    r = subprocess.run([sys.executable, "-c", _CHILD], cwd=ROOT, capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, OMP_NUM_THREADS="4"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    line = json.loads(lines[-3])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert lines[-2] == "NO_LIBFDWAVE"
    assert lines[-1] == "NO_FDWAVE_MODULE"
