"""GPU parity on an LDU matrix whose rows are not all hex-like: a seeded hex
case plus extra faces joining a few 'hub' cells to many others, so that the
widest row has more entries than the fixed-width Amul layout takes.  The
solver then uses its row-extent (CSR) Amul; every other step is the same.
Same bars as the hex cases: bit-exact Amul and DIC, 1e-10 at matched FP64
iterations, the FP64 residual bound for the mixed form."""
from functools import lru_cache

import numpy as np
import pytest

import oracle
from gpu_cases import assemble_oracle, bits, case, dev

pytestmark = pytest.mark.gpu


@lru_cache(maxsize=2)
def wide_case(centres):
    c = case(n=(10, 9, 8), jitter=0.2, permute=True, seed=21, lognormal=True)
    m = c.mesh
    uo, do = assemble_oracle(c)
    rng = np.random.default_rng(22)
    n = m.n_cells
    pairs = {(int(l), int(u)): float(a) for l, u, a in zip(m.lower, m.upper_addr, uo)}
    d = do.copy()
    scale = float(np.abs(uo).mean())
    for hub in rng.choice(n, size=3, replace=False):
        for other in rng.choice(n, size=14, replace=False):
            if other == hub:
                continue
            key = (int(min(hub, other)), int(max(hub, other)))
            if key in pairs:
                continue
            a = -0.1 * scale * (1.0 + rng.random())
            pairs[key] = a
            d[key[0]] -= a
            d[key[1]] -= a
    keys = sorted(pairs)
    lower = np.array([k[0] for k in keys], dtype=np.int32)
    upper_addr = np.array([k[1] for k in keys], dtype=np.int32)
    upper = np.array([pairs[k] for k in keys])
    width = np.bincount(lower, minlength=n) + np.bincount(upper_addr, minlength=n)
    assert width.max() > 8                                   # wider than the fixed-width layout
    from paper_2512_22215_gb300 import LduMesh
    M = LduMesh(lower, upper_addr, n, centres=m.c if centres else None)
    return lower, upper_addr, upper, d, c.b, M


@pytest.fixture(scope="module", params=[False, True], ids=["index-order", "morton"])
def wc(request):
    return wide_case(request.param)


def test_prepared_amul_bitwise(wc):
    lo, ua, up, d, b, M = wc
    M.prepare(dev(d), dev(up), 2)
    x = np.random.default_rng(23).standard_normal(len(d))
    y = M.from_internal(M.amul_prepared(M.to_internal(dev(x)))).cpu().numpy()
    assert np.array_equal(bits(y), bits(oracle.amul(lo, ua, d, up, x)))
    y1 = M.amul(dev(d), dev(up), dev(x)).cpu().numpy()
    assert np.array_equal(bits(y1), bits(oracle.amul(lo, ua, d, up, x)))


def test_dic_bitwise(wc):
    lo, ua, up, d, b, M = wc
    M.prepare(dev(d), dev(up), 2)
    rDo, bad = oracle.dic_factor(lo, ua, d, up)
    assert bad == -1
    assert np.array_equal(bits(M.read_rD().cpu().numpy()), bits(rDo))
    r = np.random.default_rng(24).standard_normal(len(d))
    w = M.precondition(dev(r), 2).cpu().numpy()
    assert np.array_equal(bits(w), bits(oracle.dic_precondition(lo, ua, up, rDo, r)))


def test_pcg_fp64_matched_iterations(wc):
    from paper_2512_22215_gb300 import SolverControls
    lo, ua, up, d, b, M = wc
    x, p = M.solve(dev(d), dev(up), dev(b), None, SolverControls(precond=2, tolerance=1e-10))
    _, po = oracle.pcg(lo, ua, d, up, b, precond=2, tol=1e-10)
    assert p["converged"] == 1 and p["status"] == 0
    assert abs(p["n_iter"] - po["n_iter"]) <= 1
    xo, _ = oracle.pcg(lo, ua, d, up, b, precond=2, tol=0.0, max_iter=p["n_iter"])
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


def test_mixed_reliable(wc):
    from paper_2512_22215_gb300 import MIXED, SolverControls
    lo, ua, up, d, b, M = wc
    x, p = M.solve(dev(d), dev(up), dev(b), None, SolverControls(precond=2, precision=MIXED, tolerance=1e-10))
    assert p["converged"] == 1 and p["status"] == 0 and p["n_outer"] >= 1
    r = b - oracle.amul(lo, ua, d, up, x.cpu().numpy())
    assert np.abs(r).sum() / np.abs(b).sum() < 1e-10


def test_gamg_matched_iterations(wc):
    """GAMG whose level 0 runs in internal order on the row-extent (CSR)
    layout, against the oracle at matched V-cycles."""
    from oracle import gamg as G
    from paper_2512_22215_gb300 import GamgSolver, SolverControls
    lo, ua, up, d, b, M = wc
    w = np.abs(up)
    S = GamgSolver(M, dev(w), smoother=1)
    assert len(S.level_cells) >= 2
    x, p = S.solve(dev(d), dev(up), dev(b), None, SolverControls(tolerance=1e-10, max_iter=500))
    assert p["converged"] == 1 and p["status"] == 0
    xo, _, _ = G.gamg(lo, ua, d, up, b, w, tol=0.0, max_iter=p["n_iter"], smoother="gs2")
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)
