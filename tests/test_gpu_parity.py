"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances. Both sides compute in FP64; they differ only in summation order
(dense DMMA tiles against CSR loops, fused RK4 combination) and in x * (1/tr)
against x / tr. One right-hand-side evaluation therefore agrees to a few ulps
of its largest term, max|f| * 1e-13 here. Over many RK4 steps the dynamics
is dissipative (omega > 0) or unitary-like (omega = 0), so rounding
differences do not grow exponentially; the trajectory bound used is
||rho_gpu - rho_oracle||_F <= 1e-10, four orders tighter than the 1e-6 the
precision form is held to.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from oracle.cpu import populations, ranking
from paper_2003_04930_gb300 import Solver, graphs
from paper_2003_04930_gb300 import qpr as Q

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04930_gb300.build import build_library
    build_library()
    assert torch.cuda.is_available()


def _pair(g, backend=Q.QPR_BACKEND_AUTO, **kw):
    return Oracle.from_edges(g, **kw), Solver.from_edges(g, backend=backend, **kw)


BACKENDS = [Q.QPR_BACKEND_DENSE, Q.QPR_BACKEND_SPARSE]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("backend", BACKENDS)
@pytest.mark.parametrize("n", [2, 16, 33, 64, 100, 150])
@pytest.mark.parametrize("omega", [0.0, 0.5, 1.0])
def test_rhs_parity(n, omega, backend):
    g = graphs.heavy_tailed(n, 40 + n) if n > 8 else graphs.erdos_renyi(n, 0.5, 1)
    o, s = _pair(g, backend, alpha=0.85, omega=omega)
    assert s.backend == backend
    rho = graphs.random_hermitian(n, 7)
    f_ref = o.rhs(rho)
    out = torch.zeros((n, n), dtype=torch.complex128, device=DEV)
    s.rhs(_dev(rho), out)
    f = out.cpu().numpy()
    scale = max(1.0, np.abs(f_ref).max())
    assert np.abs(f - f_ref).max() <= 1e-13 * scale * max(1, n / 16)
    # exact Hermiticity of the GPU right-hand side
    assert np.abs(f - f.conj().T).max() == 0.0
    r = s.residual(_dev(rho))
    assert abs(r - np.linalg.norm(f_ref)) <= 1e-12 * np.linalg.norm(f_ref)


@pytest.mark.parametrize("backend", BACKENDS)
@pytest.mark.parametrize("h_diag,dangling", [(0, 1), (1, 0), (1, 1)])
def test_rhs_parity_modes(h_diag, dangling, backend):
    g = graphs.erdos_renyi(70, 0.05, 3)  # sparse: several dangling nodes
    o, s = _pair(g, backend, alpha=0.7, omega=0.6, h_diag=h_diag, dangling=dangling)
    rho = graphs.random_density(70, 8)
    f_ref = o.rhs(rho)
    out = torch.zeros((70, 70), dtype=torch.complex128, device=DEV)
    s.rhs(_dev(rho), out)
    assert np.abs(out.cpu().numpy() - f_ref).max() <= 1e-13 * max(1.0, np.abs(f_ref).max()) * 5


@pytest.mark.parametrize("backend", BACKENDS)
def test_config1_trajectory_parity(backend):
    # N = 16 ER (p = 0.25, seed 0), alpha = 0.85, omega = 0.8, rho0 = I/N,
    # dt = 0.01 to t = 100
    g = graphs.erdos_renyi(16, 0.25, 0)
    o, s = _pair(g, backend, alpha=0.85, omega=0.8)
    rho0 = graphs.maximally_mixed(16)
    ref = o.evolve(rho0, 0.01, 10000)
    rho = _dev(rho0)
    s.evolve(rho, 0.01, 10000)
    got = rho.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-11
    assert abs(np.trace(got).real - 1.0) < 1e-14


@pytest.mark.parametrize("backend", BACKENDS)
@pytest.mark.parametrize("n", [64, 97, 200])
@pytest.mark.parametrize("omega", [0.2, 0.5, 0.8, 1.0])
def test_trajectory_parity_heavy_tailed(n, omega, backend):
    g = graphs.heavy_tailed(n, 1)
    o, s = _pair(g, backend, alpha=0.85, omega=omega)
    rho0 = graphs.random_density(n, 3, rank=2)
    ref = o.evolve(rho0, 0.01, 150)
    rho = _dev(rho0)
    s.evolve(rho, 0.01, 150)
    got = rho.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10
    assert np.abs(got - got.conj().T).max() == 0.0


def test_steady_state_parity_and_step_count():
    g = graphs.heavy_tailed(48, 2)
    o, s = _pair(g, alpha=0.85, omega=0.8)
    rho0 = graphs.maximally_mixed(48)
    ref, steps_ref, r_ref, st = o.steady_state(rho0, 0.01, 1e-8, 100000)
    assert st == 0
    rho = _dev(rho0)
    stats = s.steady_state(rho, 0.01, 1e-8, 100000)
    assert stats["converged"] == 1 and stats["residual"] < 1e-8
    assert abs(stats["steps"] - steps_ref) <= 1
    got = rho.cpu().numpy()
    if stats["steps"] == steps_ref:
        assert np.linalg.norm(got - ref) <= 1e-10
        assert abs(stats["residual"] - r_ref) <= 1e-12
    p, rank = s.populations(rho, with_rank=True)
    pr = populations(ref)
    assert np.abs(p - pr).max() <= 1e-7 * pr.max()
    np.testing.assert_array_equal(rank, ranking(p))


def test_not_converged_status_and_state():
    g = graphs.heavy_tailed(40, 5)
    o, s = _pair(g, alpha=0.85, omega=0.5)
    rho0 = graphs.maximally_mixed(40)
    rho = _dev(rho0)
    stats = s.steady_state(rho, 0.01, 1e-12, 37, check=False)
    assert stats["status"] == Q.QPR_E_NOT_CONVERGED
    assert stats["steps"] == 37 and stats["converged"] == 0
    ref = o.evolve(rho0, 0.01, 37)
    assert np.linalg.norm(rho.cpu().numpy() - ref) <= 1e-11
    assert abs(stats["residual"] - o.residual(ref)) <= 1e-12


def test_host_and_device_buffers_agree():
    g = graphs.heavy_tailed(50, 6)
    s = Solver.from_edges(g, alpha=0.85, omega=0.3)
    rho0 = graphs.random_density(50, 1)
    host = rho0.copy()
    s.evolve(host, 0.01, 40)
    dev = _dev(rho0)
    s.evolve(dev, 0.01, 40)
    np.testing.assert_array_equal(host, dev.cpu().numpy())


def test_zero_steps_returns_normalised_hermitian_part():
    g = graphs.erdos_renyi(20, 0.2, 4)
    s = Solver.from_edges(g, alpha=0.85, omega=0.3)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20)) + 20 * np.eye(20)
    h = 0.5 * (x + x.conj().T)
    d = _dev(x)
    s.evolve(d, 0.01, 0)
    np.testing.assert_allclose(d.cpu().numpy(), h / np.trace(h).real, rtol=0, atol=1e-16)


def test_no_edges_graph():
    g = graphs.erdos_renyi(30, 0.0, 0)  # every node dangles; H = 0
    o, s = _pair(g, alpha=0.85, omega=0.6)
    rho0 = graphs.random_density(30, 2)
    ref = o.evolve(rho0, 0.01, 100)
    d = _dev(rho0)
    s.evolve(d, 0.01, 100)
    assert np.linalg.norm(d.cpu().numpy() - ref) <= 1e-12


def test_unstable_dt_rejected_and_substepped():
    g = graphs.heavy_tailed(64, 9)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8, h_diag=Q.QPR_HDIAG_NEG_OUTDEG)
    dmax = s.max_stable_dt
    assert 0 < dmax < 1.0
    d = _dev(graphs.maximally_mixed(64))
    with pytest.raises(Q.QprError) as ei:
        s.evolve(d, 3.0 * dmax, 1)
    assert ei.value.status == Q.QPR_E_UNSTABLE
    stats = s.steady_state(d, 3.0 * dmax, 1e-6, 200000)
    assert stats["substeps_m"] >= 3 and stats["converged"] == 1


def test_nan_input_reported():
    g = graphs.heavy_tailed(32, 1)
    s = Solver.from_edges(g, alpha=0.85, omega=0.5)
    x = graphs.maximally_mixed(32)
    x[3, 5] = np.nan
    d = _dev(x)
    stats = s.steady_state(d, 0.01, 1e-8, 10, check=False)
    assert stats["status"] == Q.QPR_E_NONFINITE


@pytest.mark.parametrize("backend", BACKENDS)
def test_airline_size_short_trajectory(backend):
    # N = 922 heavy-tailed graph (seed 1) in the launch configuration the
    # benchmark times; a few steps against the oracle
    g = graphs.heavy_tailed(922, 1)
    o, s = _pair(g, backend, alpha=0.85, omega=0.8)
    rho0 = graphs.maximally_mixed(922)
    ref = o.evolve(rho0, 0.01, 3)
    d = _dev(rho0)
    s.evolve(d, 0.01, 3)
    got = d.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10
    assert abs(s.residual(d) - o.residual(ref)) <= 1e-11 * max(1.0, o.residual(ref))


def test_backends_agree_bitwise_independent_of_graph_chunking():
    # the number of steps per captured graph does not change the result
    g = graphs.heavy_tailed(80, 4)
    rho0 = _dev(graphs.random_density(80, 5))
    outs = []
    for gs in (0, 1, 7, 32):
        s = Solver.from_edges(g, alpha=0.85, omega=0.5, graph_steps=gs)
        r = rho0.clone()
        st = s.steady_state(r, 0.01, 1e-6, 100000)
        outs.append((st["steps"], r.cpu().numpy()))
    for st, r in outs[1:]:
        assert st == outs[0][0]
        np.testing.assert_array_equal(r, outs[0][1])


def test_profile_step_reports_positive_times():
    g = graphs.heavy_tailed(128, 3)
    s = Solver.from_edges(g, alpha=0.85, omega=0.8)
    rho = _dev(graphs.maximally_mixed(128))
    before = rho.clone()
    p = s.profile_step(rho, 0.01, 3)
    # FP64 form: a gain kernel and a fused stage kernel per stage
    assert p["product_ms"] > 0 and p["gain_ms"] > 0 and p["epilogue_ms"] == 0 and p["refresh_ms"] == 0
    assert p["launches_per_step"] == 8
    assert p["step_ms"] == pytest.approx(4 * (p["product_ms"] + p["gain_ms"]), rel=1e-9)
    assert torch.equal(rho, before)
    # mixed column-block form: SpMM (its leading CTAs form the gain) and epilogue per stage, and the refresh
    m = Solver.from_edges(g, alpha=0.85, omega=0.8, precision=Q.QPR_MIXED, backend=Q.QPR_BACKEND_SPARSE)
    assert m.sparse_form == Q.QPR_SPARSE_FORM_COLUMNS
    q = m.profile_step(rho, 0.01, 3)
    assert min(q["product_ms"], q["epilogue_ms"], q["refresh_ms"]) > 0 and q["gain_ms"] == 0
    assert q["launches_per_step"] == 8
    assert q["step_ms"] == pytest.approx(4 * (q["product_ms"] + q["epilogue_ms"]), rel=1e-9)
    assert torch.equal(rho, before)
