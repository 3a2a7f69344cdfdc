"""GPU: error paths (no fault, no hang), batched solves, the autograd adjoint
against finite differences and the dense gradient, and the full-size
workloads (128^3 and 200^3) in the benchmark's launch configuration."""
import numpy as np
import pytest
import torch

import hexmesh
import oracle
from gpu_cases import assemble_gpu, assemble_oracle, bits, case, dev, mesh_of

pytestmark = pytest.mark.gpu


def test_create_rejects_unsorted_addressing():
    from paper_2512_22215_gb300 import LduMesh, SpumaError
    lo = np.array([0, 1, 0], np.int32)
    up = np.array([1, 2, 2], np.int32)
    with pytest.raises(SpumaError) as e:
        LduMesh(lo, up, 3)
    assert e.value.status == 2
    with pytest.raises(SpumaError):
        LduMesh(np.array([1], np.int32), np.array([1], np.int32), 3)     # l == u
    with pytest.raises(SpumaError):
        LduMesh(np.array([0], np.int32), np.array([5], np.int32), 3)     # out of range


def test_device_errors_are_reported_not_trapped():
    from paper_2512_22215_gb300 import SolverControls, SpumaError, lib
    c = case(8, jitter=0.2, permute=True, seed=21, lognormal=True)
    M = mesh_of(c)
    uo, do = assemble_oracle(c)
    # negative definite matrix: the DIC pivot check fires
    with pytest.raises(SpumaError) as e:
        M.solve(dev(-do), dev(-uo), dev(c.b), None, SolverControls(precond=2))
    assert e.value.status == 6
    # NaN in b
    b = c.b.copy()
    b[5] = np.nan
    with pytest.raises(SpumaError) as e:
        M.solve(dev(do), dev(uo), dev(b), None, SolverControls(precond=2))
    assert e.value.status == 7
    # a grid barrier whose wait runs out returns a status instead of hanging
    # (32-thread blocks: the 512-cell mesh spans 16 blocks, so blocks do wait)
    lib().spuma_set_barrier_timeout_ns(0)
    try:
        _, p = M.solve(dev(do), dev(uo), dev(c.b), None, SolverControls(precond=2, block_threads=32),
                       check_status=False)
    finally:
        lib().spuma_set_barrier_timeout_ns(2_000_000_000)
    assert p["status"] == 8 and p["converged"] == 0
    # the context stays usable
    x, p = M.solve(dev(do), dev(uo), dev(c.b), None, SolverControls(precond=2, tolerance=1e-10))
    assert p["status"] == 0 and p["converged"] == 1
    # singular (zero) matrix: flagged in the report, not an error
    _, p = M.solve(dev(0 * do), dev(0 * uo), dev(c.b), None, SolverControls(precond=0))
    assert p["singular"] == 1 and p["status"] == 0


def test_empty_and_faceless_meshes():
    from paper_2512_22215_gb300 import LduMesh, SolverControls
    M = LduMesh(np.zeros(0, np.int32), np.zeros(0, np.int32), 5)
    assert M.n_levels == 1
    d = np.linspace(1, 2, 5)
    b = np.arange(1.0, 6.0)
    x, p = M.solve(dev(d), torch.zeros(0, dtype=torch.float64, device="cuda"), dev(b), None,
                   SolverControls(precond=1, tolerance=1e-14))
    assert p["n_iter"] == 1 and np.allclose(x.cpu().numpy(), b / d, rtol=1e-15)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle_per_system(precision):
    from paper_2512_22215_gb300 import BatchSolve, SolverControls
    sides = [5, 9, 12, (7, 11, 3), 16, 6]
    cs = [case(s, jitter=0.2, permute=True, seed=30 + k, lognormal=True) for k, s in enumerate(sides)]
    Ms = [mesh_of(c) for c in cs]
    ups, dgs = zip(*[assemble_oracle(c) for c in cs])
    D = [dev(d) for d in dgs]
    U = [dev(u) for u in ups]
    B = [dev(c.b) for c in cs]
    X = [torch.zeros_like(b) for b in B]
    ctl = SolverControls(precond=2, precision=precision, tolerance=1e-10)
    bs = BatchSolve(Ms, D, U, B, X, ctl, autotune=True)
    assert bs.graph_captured                   # replayed from a CUDA graph, not direct launches
    # the tuner timed a staged search: every block size that can run, then the split weights, then the grid
    assert {t["block_threads"] for t in bs.trials} >= {64, 128, 256, 512}
    assert len(bs.trials) >= 7 and bs.tuned_ms == pytest.approx(min(t["ms"] for t in bs.trials), abs=1e-3)
    bs.run()
    res = bs.results()
    first = [x.clone() for x in X]
    for k, c in enumerate(cs):
        m = c.mesh
        assert res[k]["status"] == 0 and res[k]["converged"] == 1
        x = X[k].cpu().numpy()
        if precision == 0:
            xo, po = oracle.pcg(m.lower, m.upper_addr, dgs[k], ups[k], c.b, precond=2, tol=0.0,
                                max_iter=res[k]["n_iter"])
            assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)
        r = c.b - oracle.amul(m.lower, m.upper_addr, dgs[k], ups[k], x)
        assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-10
        assert res[k]["true_rel_residual_l2"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(c.b), rel=1e-12)
    for x in X:
        x.zero_()
    bs.run()                                   # graph replay: same answers bit for bit
    for a, b in zip(first, X):
        assert torch.equal(a, b)


def test_batch_without_graph():
    """The direct-launch replay (no graph) gives the graph's answers bit for bit."""
    from paper_2512_22215_gb300 import BatchSolve, SolverControls
    cs = [case(s, jitter=0.2, permute=True, seed=35 + k, lognormal=True) for k, s in enumerate([7, 10, 5])]
    Ms = [mesh_of(c) for c in cs]
    ups, dgs = zip(*[assemble_oracle(c) for c in cs])
    D, U, B = [dev(d) for d in dgs], [dev(u) for u in ups], [dev(c.b) for c in cs]
    ctl = SolverControls(precond=2, tolerance=1e-10, block_threads=128)
    X1 = [torch.zeros_like(b) for b in B]
    g = BatchSolve(Ms, D, U, B, X1, ctl, autotune=False)
    assert g.graph_captured and g.tuned_ms == -1.0 and g.trials == []
    g.run()
    X2 = [torch.zeros_like(b) for b in B]
    d = BatchSolve(Ms, D, U, B, X2, ctl, autotune=False, graph=False)
    assert not d.graph_captured
    d.run()
    torch.cuda.synchronize()
    for a, b in zip(X1, X2):
        assert torch.equal(a, b)


@pytest.mark.slow
def test_batch_64_systems_log_uniform():
    """The batched workload: 64 jittered, permuted hex blocks with cell counts
    log-uniform in 1e4..5e5 (sides from hexmesh.batch_sizes, seed 5; 8.2M
    cells), FP64 and mixed, tuned and replayed from a CUDA graph.  Every system
    reaches the oracle's FP64 residual 1e-8; FP64 systems of at most 64^3
    cells match the oracle's PCG at the same iteration count to 1e-8.  That
    bound is the arithmetic's, not the kernel's: two FP64 PCG runs on the CPU
    that differ only in the order of their dot-product sums (the oracle's
    sequential sums against pairwise ones, with the oracle's Amul and DIC)
    drift apart by 8.9e-10 on this batch's 23^3 system (seed 504, 96
    iterations) and 8.1e-10 at 62^3 (seed 500, 248 iterations); the GPU's
    fixed reduction tree is such an order."""
    from paper_2512_22215_gb300 import MIXED, BatchSolve, LduMesh, SolverControls
    sides = hexmesh.batch_sizes(64, seed=5)
    cs = [hexmesh.pressure_case(n, jitter=0.2, permute=True, seed=500 + k, lognormal_gamma=True)
          for k, n in enumerate(sides)]
    assert sum(c.mesh.n_cells for c in cs) > 8_000_000
    Ms = [LduMesh(c.mesh.lower, c.mesh.upper_addr, c.mesh.n_cells, centres=c.mesh.c) for c in cs]
    ups, dgs = zip(*[assemble_oracle(c) for c in cs])
    D, U, B = [dev(d) for d in dgs], [dev(u) for u in ups], [dev(c.b) for c in cs]
    for precision in (0, MIXED):
        X = [torch.zeros_like(b) for b in B]
        bs = BatchSolve(Ms, D, U, B, X, SolverControls(precond=2, precision=precision, tolerance=1e-8))
        assert bs.graph_captured
        bs.run()
        res = bs.results()
        for k, c in enumerate(cs):
            m = c.mesh
            assert res[k]["status"] == 0 and res[k]["converged"] == 1, (k, res[k])
            x = X[k].cpu().numpy()
            r = c.b - oracle.amul(m.lower, m.upper_addr, dgs[k], ups[k], x)
            assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-8
            assert res[k]["true_rel_residual_l2"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(c.b),
                                                                   rel=1e-12)
            if precision == 0 and m.n_cells <= 64 ** 3:
                xo, _ = oracle.pcg(m.lower, m.upper_addr, dgs[k], ups[k], c.b, precond=2, tol=0.0,
                                   max_iter=res[k]["n_iter"])
                assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo), (k, res[k]["n_iter"])


def test_autograd_dense_gradient_8cubed():
    from paper_2512_22215_gb300 import SolverControls, pressure_solve
    c = case(8, jitter=0.2, permute=True, seed=40, lognormal=True, target=True)
    m = c.mesh
    M = mesh_of(c)
    uo, do = assemble_oracle(c)
    up = dev(uo).requires_grad_(True)
    dg = dev(do).requires_grad_(True)
    b = dev(c.b).requires_grad_(True)
    x = pressure_solve(M, up, dg, b, SolverControls(precond=2, tolerance=1e-14))
    loss = 0.5 * ((x - dev(c.x_t)) ** 2).sum()
    loss.backward()
    A = np.zeros((m.n_cells, m.n_cells))
    A[np.arange(m.n_cells), np.arange(m.n_cells)] = do
    A[m.lower, m.upper_addr] = uo
    A[m.upper_addr, m.lower] = uo
    xs = np.linalg.solve(A, c.b)
    lam = np.linalg.solve(A, xs - c.x_t)
    G = -np.outer(lam, xs)
    assert np.allclose(b.grad.cpu().numpy(), lam, rtol=1e-9, atol=1e-12 * np.abs(lam).max())
    assert np.allclose(up.grad.cpu().numpy(), G[m.lower, m.upper_addr] + G[m.upper_addr, m.lower], rtol=1e-8,
                       atol=1e-11 * np.abs(G).max())
    assert np.allclose(dg.grad.cpu().numpy(), np.diag(G), rtol=1e-8, atol=1e-11 * np.abs(G).max())


@pytest.mark.parametrize("n", [64, pytest.param(128, marks=pytest.mark.slow)])
def test_autograd_finite_differences(n):
    """32 random directions, central differences with step 1e-6 (relative to the
    perturbed quantity), FP64 solves to 1e-14; agreement to 1e-6 relative."""
    from paper_2512_22215_gb300 import SolverControls, pressure_solve
    c = case(n, jitter=0.2, permute=True, seed=4, lognormal=True, target=True)
    M = mesh_of(c)
    uo, do = assemble_oracle(c)
    ctl = SolverControls(precond=2, tolerance=1e-14, max_iter=3000)
    xt = dev(c.x_t)

    def L(up, dg, b):
        with torch.no_grad():
            x = pressure_solve(M, up, dg, b, ctl)
        return 0.5 * float(((x - xt) ** 2).sum())

    up = dev(uo).requires_grad_(True)
    dg = dev(do)
    b = dev(c.b).requires_grad_(True)
    x = pressure_solve(M, up, dg, b, ctl)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    gb, gu = b.grad.double(), up.grad.double()
    rng = np.random.default_rng(123)
    h = 1e-6
    for _ in range(32):
        vb = dev(rng.standard_normal(c.mesh.n_cells))
        vu = dev(rng.standard_normal(c.mesh.n_faces) * np.abs(uo))
        fd_b = (L(up.detach(), dg, b.detach() + h * vb) - L(up.detach(), dg, b.detach() - h * vb)) / (2 * h)
        fd_u = (L(up.detach() + h * vu, dg, b.detach()) - L(up.detach() - h * vu, dg, b.detach())) / (2 * h)
        assert fd_b == pytest.approx(float((gb * vb).sum()), rel=1e-6)
        assert fd_u == pytest.approx(float((gu * vu).sum()), rel=1e-6)


@pytest.mark.slow
@pytest.mark.parametrize("n,seed", [(128, 2), (200, 3)])
def test_full_size_workloads(n, seed):
    """The benchmark workloads: jittered, permuted, log-normal gamma.  Whole-array
    bit-exactness of assembly, Amul and the DIC factor; matched-iteration FP64
    PCG parity over the first iterations; FP64 and mixed solves to 1e-8 checked
    with the oracle's FP64 residual."""
    from paper_2512_22215_gb300 import MIXED, SolverControls
    c = case(n, jitter=0.2, permute=True, seed=seed, lognormal=True)
    m = c.mesh
    M = mesh_of(c, centres=True)
    up, dg = assemble_gpu(M, c)
    uo, do = assemble_oracle(c)
    assert np.array_equal(bits(up.cpu().numpy()), bits(uo)) and np.array_equal(bits(dg.cpu().numpy()), bits(do))
    x = np.random.default_rng(1).standard_normal(m.n_cells)
    assert np.array_equal(bits(M.amul(dg, up, dev(x)).cpu().numpy()),
                          bits(oracle.amul(m.lower, m.upper_addr, do, uo, x)))
    M.prepare(dg, up, 2)
    rDo, _ = oracle.dic_factor(m.lower, m.upper_addr, do, uo)
    assert np.array_equal(bits(M.read_rD().cpu().numpy()), bits(rDo))
    xg, p = M.solve(dg, up, dev(c.b), None, SolverControls(precond=2, tolerance=0.0, max_iter=4))
    xo, _ = oracle.pcg(m.lower, m.upper_addr, do, uo, c.b, precond=2, tol=0.0, max_iter=4)
    assert np.linalg.norm(xg.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
    nfac = np.abs(c.b).sum() + 1e-20
    for precond, precision in [(2, 0), (1, 0), (2, MIXED)]:
        xs, p = M.solve(dg, up, dev(c.b), None, SolverControls(precond=precond, precision=precision, tolerance=1e-8))
        assert p["converged"] == 1 and p["status"] == 0
        r = c.b - oracle.amul(m.lower, m.upper_addr, do, uo, xs.cpu().numpy())
        assert np.abs(r).sum() / nfac < 1e-8
