"""Child process of test_gpu_env_paths.py: runs the bit-exact DIC checks, the
FP64 / mixed solves and GAMG on one seeded case under whatever SPUMA_* variables
the parent set (the library reads them once per process), and prints one
JSON line with the comparisons against the oracle."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
from gpu_cases import assemble_oracle, bits, case, dev, mesh_of  # noqa: E402


def main():
    from paper_2512_22215_gb300 import MIXED, SolverControls
    c = case(n=(23, 17, 13), jitter=0.2, permute=True, seed=61, lognormal=True)
    m = c.mesh
    M = mesh_of(c, centres=True)
    uo, do = assemble_oracle(c)
    out = {"levels": M.n_levels}
    M.prepare(dev(do), dev(uo), 2)
    rDo, bad = oracle.dic_factor(m.lower, m.upper_addr, do, uo)
    out["rD_bitwise"] = bool(bad == -1 and np.array_equal(bits(M.read_rD().cpu().numpy()), bits(rDo)))
    r = np.random.default_rng(62).standard_normal(m.n_cells)
    w = M.precondition(dev(r), 2).cpu().numpy()
    out["precondition_bitwise"] = bool(np.array_equal(bits(w), bits(oracle.dic_precondition(m.lower, m.upper_addr,
                                                                                               uo, rDo, r))))
    for threads in (1024, 64):
        x, p = M.solve(dev(do), dev(uo), dev(c.b), None,
                       SolverControls(precond=2, tolerance=1e-10, max_iter=5000, block_threads=threads))
        xo, po = oracle.pcg(m.lower, m.upper_addr, do, uo, c.b, precond=2, tol=0.0, max_iter=p["n_iter"])
        out[f"fp64_{threads}"] = {"converged": p["converged"], "status": p["status"], "n_iter": p["n_iter"],
                                  "rel_err": float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo))}
    x, p = M.solve(dev(do), dev(uo), dev(c.b), None,
                   SolverControls(precond=2, precision=MIXED, tolerance=1e-10, max_iter=5000))
    res = c.b - oracle.amul(m.lower, m.upper_addr, do, uo, x.cpu().numpy())
    out["mixed"] = {"converged": p["converged"], "status": p["status"],
                    "oracle_residual": float(np.abs(res).sum() / np.abs(c.b).sum())}
    from oracle import gamg as G
    from paper_2512_22215_gb300 import GamgSolver
    wts = np.abs(uo)
    for smoother, name in ((0, "richardson"), (1, "gs2")):
        S = GamgSolver(M, dev(wts), smoother=smoother)
        x, p = S.solve(dev(do), dev(uo), dev(c.b), None, SolverControls(tolerance=1e-10, max_iter=500))
        xo, _, _ = G.gamg(m.lower, m.upper_addr, do, uo, c.b, wts, tol=0.0, max_iter=p["n_iter"], smoother=name)
        out[f"gamg_{name}"] = {"converged": p["converged"], "status": p["status"], "levels": len(S.level_cells),
                               "rel_err": float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo))}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
