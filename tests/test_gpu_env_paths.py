"""The solvers' measurement overrides (SPUMA_SWEEP=0: DIC levels strided over
the blocks; SPUMA_TAIL_ROWS=0: no small last levels on the first block;
SPUMA_SOLVE_BLOCKS_PER_SM=1; SPUMA_GAMG_FUSE_SCALE_ROWS: GAMG's correction
scaling inside the first smoothing sweep; SPUMA_GAMG_ORDER=inherited: GAMG's
middle levels stored in the inherited order) change how a solve runs, never
what it computes.  The library reads them once per process, so each setting
runs in a child process (tests/env_path_child.py) that compares with the
oracle: DIC factor and preconditioner bit for bit, FP64 PCG at matched
iterations to 1e-10 at two block sizes, the mixed form's FP64 residual below
1e-10, GAMG (Richardson and two-stage Gauss-Seidel) at matched V-cycles to
1e-8."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SETTINGS = [{}, {"SPUMA_SWEEP": "0"}, {"SPUMA_TAIL_ROWS": "0"}, {"SPUMA_SWEEP": "0", "SPUMA_TAIL_ROWS": "0"},
            {"SPUMA_SOLVE_BLOCKS_PER_SM": "1"}, {"SPUMA_GAMG_FUSE_SCALE_ROWS": "1000000"},
            {"SPUMA_GAMG_ORDER": "inherited"}]
IDS = ["default", "strided-levels", "no-tail", "strided-no-tail", "one-block-per-sm", "gamg-fused-scaling",
       "gamg-inherited-order"]


@pytest.mark.parametrize("env", SETTINGS, ids=IDS)
def test_override_keeps_results(env):
    e = {k: v for k, v in os.environ.items() if not k.startswith("SPUMA_")}
    e.update(env)
    e["PYTHONPATH"] = ROOT + os.pathsep + e.get("PYTHONPATH", "")
    run = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "env_path_child.py")], cwd=ROOT, env=e,
                         capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stderr[-2000:]
    out = json.loads(run.stdout.strip().splitlines()[-1])
    assert out["levels"] > 1
    assert out["rD_bitwise"] and out["precondition_bitwise"]
    for threads in (1024, 64):
        r = out[f"fp64_{threads}"]
        assert r["converged"] == 1 and r["status"] == 0
        assert r["rel_err"] <= 1e-10
    assert out["mixed"]["converged"] == 1 and out["mixed"]["status"] == 0
    assert out["mixed"]["oracle_residual"] < 1e-10
    for name in ("richardson", "gs2"):
        r = out[f"gamg_{name}"]
        assert r["converged"] == 1 and r["status"] == 0 and r["levels"] >= 3
        assert r["rel_err"] <= 1e-8
