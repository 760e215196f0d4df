"""The remaining workloads at full size, in the launch configurations a user runs them with.

  * single energy: 40 x 40 oscillator functions (N = 3200), eps_i = 1 eV, FP64 GMRES with the
    Jacobi preconditioner to 1e-10 (the plain FP64 solve);
  * uneven batch: 80 x 80 (N = 12,800), 128 incident energies on (0, 4] eV x the 4 lowest
    initial levels x 2 partial waves = 1024 systems of different difficulty, then cross
    sections and the EELS spectrum on a 1 meV energy-loss grid;
  * adjoint: 40 x 40 with the cubic and bilinear extra couplings, 256 energies on (0, 3] eV,
    the 10 lowest final levels, all 19 parameters.

Every solution is checked by the oracle in complex128 (true residual with the oracle's sparse
A; cross sections, EELS and gradients from sparse or dense LU) on the systems or energies the
oracle can afford, and the full-size gradient against central differences of the GPU loss.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as w  # noqa: E402
from oracle import vibronic as o  # noqa: E402

pytestmark = pytest.mark.gpu

TARGET_SEED = 2307134831  # the adjoint workload's target cross sections


@pytest.fixture(scope="module")
def vbk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2307_13483_gb300 as lib

    return lib


def test_single_energy_fp64_gmres(vbk):
    spec = w.WORKLOADS["ci2d_single"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    model = vbk.Model(desc)
    assert model.N == 3200
    opts = vbk.vbk_default_opts(method="gmres", precision="fp64", precond_span=0, tol=1e-10, restart=64, max_refine=400)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    assert all(s["status"] == "converged" for s in stats)
    psi_h = psi.cpu().numpy()
    E = o.total_energy(desc, eps[0], vi[0])
    for mu in range(model.n_mu):
        res = o.relative_residual(desc, E, psi_h[0, 0, mu], o.phi(desc, E, vi[0], mu))
        assert res <= 1e-10 * 1.05, (mu, res)
    vf = o.open_levels(desc, E)
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf).cpu().numpy()
    ref, _ = o.cross_sections(desc, eps, vi, vf)
    big = ref > 1e-6 * ref.max()
    np.testing.assert_allclose(sig[big], ref[big], rtol=1e-8)


def test_uneven_batch_full_size(vbk):
    spec = w.WORKLOADS["ci2d_uneven"]
    desc, eps = spec["model"](), spec["eps"]
    vi = w.lowest_levels(desc, 4)
    model = vbk.Model(desc)
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=0, tol=1e-8)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    assert len(stats) == 1024
    assert all(s["status"] == "converged" for s in stats)
    its = np.array([s["iterations"] for s in stats])
    assert its.min() < its.max()
    psi_h = psi.cpu().numpy()
    for e in range(0, eps.size, 4):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, eps[e], v)
            A = o.a_matrix(desc, E)
            for mu in range(2):
                rhs = o.phi(desc, E, v, mu)
                res = np.linalg.norm(rhs - A @ psi_h[e, i, mu]) / np.linalg.norm(rhs)
                assert res <= 1e-8 * 1.05, (e, i, mu, res)
    # cross sections and the EELS spectrum (1 meV loss grid) of sampled energies
    vf = w.lowest_levels(desc, 24)
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf)
    de = np.arange(0.0, 4.0, 0.001)
    S = vbk.vbk_eels(model, vi, vf, sig, de).cpu().numpy()
    sig = sig.cpu().numpy()
    sample = [5, 64, 127]
    ref, _ = o.cross_sections(desc, eps[sample], vi, vf)
    big = ref > 1e-6 * ref.max()
    np.testing.assert_allclose(sig[sample][big], ref[big], rtol=5e-6)
    for i, v in enumerate(vi):
        S_ref = o.eels(desc, eps[sample], v, vf, ref[:, i, :], de)
        np.testing.assert_allclose(S[sample, i], S_ref, rtol=5e-6, atol=1e-6 * np.abs(S_ref).max())


def _adjoint_setup(vbk):
    spec = w.WORKLOADS["ci2d_adjoint"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    vf = w.lowest_levels(desc, 10)
    nt = len(desc["terms"])
    thetas = list(range(nt)) + list(range(nt, nt + 2 * len(desc["channels"])))
    target = np.random.default_rng(TARGET_SEED).uniform(0.0, 1.0, (eps.size, len(vf)))
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", tol=1e-10, max_refine=100)
    return desc, eps, vi, vf, thetas, target, opts


def test_adjoint_full_size_sampled(vbk):
    """Gradient contributions of sampled energies (dL/dsigma zero elsewhere) against the
    oracle's dense-LU adjoint, with the forward and adjoint solves over all 256 energies."""
    desc, eps, vi, vf, thetas, target, opts = _adjoint_setup(vbk)
    assert len(thetas) == 19
    model = vbk.Model(desc)
    psi, st = vbk.vbk_solve(model, eps, vi, opts)
    assert all(s["status"] == "converged" for s in st)
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf)
    sample = [17, 140, 251]
    mask = torch.zeros_like(sig)
    mask[sample] = 1.0
    tgt = torch.tensor(target[:, None, :], device="cuda")
    dlds = 2.0 * (sig - tgt) * mask
    g, stats = vbk.vbk_solve_adjoint(model, eps, vi, psi, vf, dlds, thetas, opts)
    assert all(s["status"] in ("converged", "zero_rhs") for s in stats)
    g_ref = o.loss_gradient_adjoint(desc, eps[sample], vi[0], vf, target[sample], thetas)
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-9 * np.abs(g_ref).max())


def test_adjoint_full_size_matches_finite_differences(vbk):
    """All 256 energies weighted: the adjoint gradient in three parameter directions against
    central differences of the loss evaluated by GPU forward solves."""
    desc, eps, vi, vf, thetas, target, opts = _adjoint_setup(vbk)
    tgt = torch.tensor(target[:, None, :], device="cuda")

    def loss_and_sig(d):
        m = vbk.Model(d)
        psi, st = vbk.vbk_solve(m, eps, vi, opts)
        assert all(s["status"] == "converged" for s in st)
        sig = vbk.vbk_cross_sections(m, eps, vi, psi, vf)
        return float(((sig - tgt) ** 2).sum()), m, psi, sig

    _, model, psi, sig = loss_and_sig(desc)
    g, _ = vbk.vbk_solve_adjoint(model, eps, vi, psi, vf, 2.0 * (sig - tgt), thetas, opts)
    nt = len(desc["terms"])
    for k in (2, nt - 1, nt + 1):  # a coupling, a cubic term, a continuum range parameter
        p0 = o.get_parameter(desc, thetas[k])
        h = 1e-5 * max(1.0, abs(p0))
        lp = loss_and_sig(o.with_parameter(desc, thetas[k], p0 + h))[0]
        lm = loss_and_sig(o.with_parameter(desc, thetas[k], p0 - h))[0]
        fd = (lp - lm) / (2 * h)
        assert abs(g[k] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, g[k], fd)


def test_resident_mixed_cocg_at_tol_1e12_near_resonances(vbk):
    """How far the resident path's double-float refinement carries: FP32 COCG inside double-float
    residuals (resident = 1) at tol 1e-12 on the 80 x 80 model, at the two energies where the
    oracle's |psi| / |Phi| peaks on a 0.02 eV scan of 2.3..2.9 eV (one per partial wave: the
    resonances, where A is closest to singular), near threshold and at 3 eV.  The oracle's
    complex128 residual of the returned psi must meet the tolerance and sigma must match LU."""
    desc = w.ci2d_model(80)
    vi = [[0, 0]]
    scan = np.arange(2.30, 2.9001, 0.02)
    amp = np.zeros((scan.size, 2))
    for k, e in enumerate(scan):
        E = o.total_energy(desc, e, vi[0])
        rhs = [o.phi(desc, E, vi[0], mu) for mu in range(2)]
        ps = o.solve_many(desc, E, rhs)
        amp[k] = [np.linalg.norm(ps[:, mu]) / np.linalg.norm(rhs[mu]) for mu in range(2)]
    peaks = sorted({float(scan[np.argmax(amp[:, mu])]) for mu in range(2)})
    eps = np.array([0.05] + peaks + [3.0])
    model = vbk.Model(desc)
    tol = 1e-12
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=0, tol=tol, resident=1, max_refine=100)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    assert all(s["status"] == "converged" for s in stats), [s for s in stats]
    psi_h = psi.cpu().numpy()
    vf = o.open_levels(desc, o.total_energy(desc, float(eps[-1]), vi[0]))
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf).cpu().numpy()
    ref, _ = o.cross_sections(desc, eps, vi, vf)
    for e, ei in enumerate(eps):
        E = o.total_energy(desc, ei, vi[0])
        A = o.a_matrix(desc, E)
        for mu in range(2):
            rhs = o.phi(desc, E, vi[0], mu)
            res = np.linalg.norm(rhs - A @ psi_h[e, 0, mu]) / np.linalg.norm(rhs)
            assert res <= 1.05 * tol, (ei, mu, res)
    big = ref > 1e-6 * ref.max()
    np.testing.assert_allclose(sig[big], ref[big], rtol=1e-8)
