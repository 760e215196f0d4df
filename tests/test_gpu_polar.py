"""The polar bending basis on the GPU (Sec. III.C, CO2 paragraph): the CO2-like model with its
2D bend in circular oscillator quanta (the polar eigenfunctions of the 2D isotropic
oscillator) and couplings up to fourth order written as ladder-operator terms, through the
C ABI against the oracle:

* every matvec kernel variant, FP64 and FP32, against the oracle's sparse A;
* the states x 2D-bend block preconditioner (the paper's choice for CO2) against the oracle's
  block-diagonal section of A;
* solves (COCG and GMRES, FP64 and mixed, Jacobi and the states x bend blocks): true
  residual by the oracle, cross sections against LU;
* the adjoint gradient in ladder-term coefficients against the oracle's dense-LU adjoint.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as w  # noqa: E402
from oracle import vibronic as o  # noqa: E402

pytestmark = pytest.mark.gpu

SPAN_STATES_BEND = 0x1 | 0x4 | 0x8  # d, n_+, n_-


@pytest.fixture(scope="module")
def vbk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2307_13483_gb300 as lib

    return lib


def _small():
    return w.co2_polar_model(basis=(4, 6, 5, 3))  # ragged: n_+ and n_- truncated differently


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("variant", list(range(20)))  # VBK_MATVEC_NVARIANTS
def test_polar_matvec_parity(vbk, precision, variant):
    desc = _small()
    model = vbk.Model(desc)
    rng = np.random.default_rng(3)
    E = np.array([1.4, 3.2, 4.6])
    x = rng.standard_normal((E.size, 3, model.N)) + 1j * rng.standard_normal((E.size, 3, model.N))
    try:
        y = vbk.vbk_matvec(model, E, torch.tensor(x, device="cuda"), precision=0 if precision == "fp64" else 1,
                           variant=variant).cpu().numpy()
    except vbk.VbkError as err:
        if err.code == 1 and "variant not available" in str(err):
            pytest.skip("variant does not fit this model / precision")
        raise
    tol = 1e-13 if precision == "fp64" else 2e-6
    for e in range(E.size):
        A = o.a_matrix(desc, E[e])
        for k in range(3):
            ref = A @ x[e, k]
            assert np.linalg.norm(y[e, k] - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("span", [0, 0x1, SPAN_STATES_BEND, 0x1 | 0x4])
def test_polar_block_preconditioner_parity(vbk, precision, span):
    desc = _small()
    model = vbk.Model(desc)
    rng = np.random.default_rng(4)
    E = 3.3
    r = rng.standard_normal((1, 2, model.N)) + 1j * rng.standard_normal((1, 2, model.N))
    z = vbk.vbk_precond_apply(model, [E], torch.tensor(r, device="cuda"), span,
                              precision=0 if precision == "fp64" else 1).cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 5e-5
    for k in range(2):
        ref = o.precond_apply(desc, E, span, r[0, k])
        assert np.linalg.norm(z[0, k] - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("method,precision,span", [("cocg", "fp64", SPAN_STATES_BEND), ("cocg", "mixed", 0),
                                                   ("gmres", "mixed", SPAN_STATES_BEND), ("gmres", "fp64", 0),
                                                   ("cocg", "mixed", SPAN_STATES_BEND)])
def test_polar_solve_parity(vbk, method, precision, span):
    desc = _small()
    model = vbk.Model(desc)
    eps = np.array([0.7, 2.1, 3.0])
    vi = [[0, 0, 0, 0], [0, 1, 0, 0]]
    opts = vbk.vbk_default_opts(method=method, precision=precision, precond_span=span, tol=1e-10, restart=60,
                                max_iter=40000, max_refine=400)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    psi = psi.cpu().numpy()
    nmu = model.n_mu
    for e, ei in enumerate(eps):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, ei, v)
            A = o.a_matrix(desc, E)
            for mu in range(nmu):
                st = stats[(e * len(vi) + i) * nmu + mu]
                rhs = o.phi(desc, E, v, mu)
                if not np.any(rhs):
                    assert st["status"] == "zero_rhs"
                    continue
                assert st["status"] == "converged", st
                res = np.linalg.norm(rhs - A @ psi[e, i, mu]) / np.linalg.norm(rhs)
                assert res <= 1.05e-10, (e, i, mu, res)
    vf = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 1, 1, 0]]
    sig = vbk.vbk_cross_sections(model, eps, vi, torch.tensor(psi, device="cuda"), vf).cpu().numpy()
    ref, _ = o.cross_sections(desc, eps, vi, vf)
    big = ref > 1e-6 * ref.max()
    np.testing.assert_allclose(sig[big], ref[big], rtol=1e-8)


def test_polar_model_at_larger_basis(vbk):
    """12 x 14 x 14 x 6 circular-quanta basis (N = 42,336) at 3 eV, three partial waves, FP64
    COCG with the states x 2D-bend blocks: true residuals by the oracle."""
    desc = w.co2_polar_model(basis=(12, 14, 14, 6))
    model = vbk.Model(desc)
    assert model.N == 3 * 12 * 14 * 14 * 6
    eps, vi = np.array([3.0]), [[0, 0, 0, 0]]
    opts = vbk.vbk_default_opts(method="cocg", precision="fp64", precond_span=SPAN_STATES_BEND, tol=1e-8,
                                max_iter=20000, max_refine=100)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    assert all(s["status"] == "converged" for s in stats), stats
    psi = psi.cpu().numpy()
    E = o.total_energy(desc, 3.0, vi[0])
    A = o.a_matrix(desc, E)
    for mu in range(3):
        rhs = o.phi(desc, E, vi[0], mu)
        assert np.linalg.norm(rhs - A @ psi[0, 0, mu]) / np.linalg.norm(rhs) <= 1.05e-8


def test_polar_adjoint_in_ladder_coefficients(vbk):
    """Gradient of a cross-section loss in coefficients of ladder terms (a rho^2 part, a fourth-
    order term, the Renner-Teller and Sigma-Pi couplings) against the dense-LU adjoint."""
    desc = w.co2_polar_model(basis=(3, 4, 4, 2))
    model = vbk.Model(desc)
    eps, vi = np.array([1.8, 3.4]), [[0, 0, 0, 0]]
    vf = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0]]
    ladder = [k for k, t in enumerate(desc["terms"]) if any(t.get("raise", [])) or any(t.get("lower", []))]
    thetas = [ladder[0], ladder[1], ladder[5]] + [k for k, t in enumerate(desc["terms"]) if t["d"] != t["dp"]][:3]
    target = np.full((eps.size, len(vf)), 0.3)
    opts = vbk.vbk_default_opts(method="cocg", precision="fp64", tol=1e-12, max_refine=100)
    psi, st = vbk.vbk_solve(model, eps, vi, opts)
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf)
    dlds = 2.0 * (sig - torch.tensor(target[:, None, :], device="cuda"))
    g, _ = vbk.vbk_solve_adjoint(model, eps, vi, psi, vf, dlds, thetas, opts)
    g_ref = o.loss_gradient_adjoint(desc, eps, vi[0], vf, target, thetas)
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-9 * np.abs(g_ref).max())
