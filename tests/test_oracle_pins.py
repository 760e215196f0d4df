"""Pins of the CPU oracle against facts fixed independently of its own code.

Each test names what it pins and why a plausible mistake (a dropped term, a wrong
sign, index or factor, a transposed Kronecker product) would fail it:

* oscillator matrices: eigenvalues of the truncated q are the Gauss-Hermite nodes;
  <k|q^2|k> = k + 1/2 and <k|q^2|k+2> = sqrt((k+1)(k+2))/2 (textbook values);
* H_0 + kappa q and H_0 + gamma q^2 reproduce the displaced (-kappa^2/2omega) and
  stiffened (omega' = sqrt(omega(omega+2 gamma))) oscillator spectra;
* two states coupled by lambda q_u with equal energies give the displaced spectrum
  -lambda^2/2omega_u (pins the off-diagonal block placement);
* the level shift equals principal-value quadrature of its defining integral (Eq. IntF);
* A is complex symmetric, not Hermitian, and its anti-Hermitian part is exactly
  pi * sum over open levels of Phi Phi^T (Eqs. F_gen, Amatrix);
* flux conservation (optical theorem) in the truncated basis;
* without q-dependent terms the solution is the closed form Phi / diagonal;
* a model without q_u terms decouples into 1D problems at shifted energies,
  each solved by a separately built dense 1D matrix;
* the EELS sum integrates to the sum of the cross sections (unit-area Gaussian);
* one EELS line has its peak at the energy loss E_vf - E_vi, the peak height of a unit-area
  Gaussian of 10 meV FWHM, and half that height 5 meV either side (a FWHM used as the
  standard deviation, or a line on the wrong side of the elastic peak, fails);
* at the energy where the real part of a one-channel diagonal A vanishes, T = -i/pi and the
  cross section is the s-wave unitarity limit 4 pi / k^2 (in bohr^2, eps_i = k^2 / 2 hartree):
  this pins the prefactor of the cross section (a slip to pi^2, or eps_i in the wrong unit,
  fails), and |1 - 2 pi i T| = 1 holds at every energy of that model (elastic unitarity).
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.optimize as so

from oracle import vibronic as o
import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- oscillator matrices
@pytest.mark.parametrize("n", [1, 2, 5, 12, 40])
def test_q_eigenvalues_are_gauss_hermite_nodes(n):
    nodes, _ = np.polynomial.hermite.hermgauss(n)
    ev = np.linalg.eigvalsh(o.q_matrix(n))
    np.testing.assert_allclose(np.sort(ev), np.sort(nodes), atol=1e-12)


def test_q_squared_textbook_elements():
    n = 10
    q2 = o.q_power(n, 2)
    for k in range(n - 2):
        assert q2[k, k] == pytest.approx(k + 0.5, abs=1e-14)
        assert q2[k, k + 2] == pytest.approx(math.sqrt((k + 1) * (k + 2)) / 2, abs=1e-14)
        assert q2[k, k + 1] == 0.0
    # truncated product (PqP)(PqP): the last diagonal element keeps only the downward path
    assert q2[n - 1, n - 1] == pytest.approx((n - 1) / 2, abs=1e-14)


def _one_mode_model(n, omega, terms, channels=None):
    return {"n_states": 1, "modes": [{"name": "x", "omega": omega, "n": n}], "terms": terms,
            "channels": channels or [{"d": 0, "mu": 0, "a": 0.0, "b": 1.0, "l": 0}]}


def test_displaced_oscillator_spectrum():
    omega, kappa, n = 0.21, -0.17, 60
    m = _one_mode_model(n, omega, [{"d": 0, "dp": 0, "coef": kappa, "pow": [1]}])
    E = 0.7
    A = o.a_matrix(m, E).toarray()
    H = E * np.eye(A.shape[0]) - A  # a = 0: no continuum, so H = H_0 + U
    ev = np.sort(np.linalg.eigvals(H).real)[:8]
    np.testing.assert_allclose(ev, omega * (np.arange(8) + 0.5) - kappa ** 2 / (2 * omega), atol=1e-10)


def test_stiffened_oscillator_spectrum():
    omega, gamma, n = 0.19, 0.07, 80
    m = _one_mode_model(n, omega, [{"d": 0, "dp": 0, "coef": gamma, "pow": [2]}])
    A = o.a_matrix(m, 1.0).toarray()
    H = np.eye(A.shape[0]) - A
    ev = np.sort(np.linalg.eigvals(H).real)[:6]
    wp = math.sqrt(omega * (omega + 2 * gamma))
    np.testing.assert_allclose(ev, wp * (np.arange(6) + 0.5), atol=1e-9)


def test_two_state_linear_coupling_spectrum():
    wg, wu, lam, n = 0.25, 0.13, 0.11, 50
    m = {"n_states": 2, "modes": [{"name": "g", "omega": wg, "n": 3}, {"name": "u", "omega": wu, "n": n}],
         "terms": [{"d": 0, "dp": 1, "coef": lam, "pow": [0, 1]}],
         "channels": [{"d": 0, "mu": 0, "a": 0.0, "b": 1.0, "l": 0}, {"d": 1, "mu": 1, "a": 0.0, "b": 1.0, "l": 0}]}
    A = o.a_matrix(m, 2.0).toarray()
    H = 2.0 * np.eye(A.shape[0]) - A
    ev = np.sort(np.linalg.eigvals(H).real)[:4]
    shift = wg * 0.5 - lam ** 2 / (2 * wu)
    np.testing.assert_allclose(ev, shift + wu * np.array([0.5, 0.5, 1.5, 1.5]), atol=1e-9)


# ---------------------------------------------------------------------- level shift
def _shift_by_quadrature(eps, a, b, l):
    f = lambda x: a / (2 * math.pi) * x ** (l + 0.5) * math.exp(-b * x)
    top = 60.0 / b + 10.0 * (l + 1)
    if eps > 0:
        pv = -si.quad(f, 0.0, top, weight="cauchy", wvar=eps, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    else:
        pv = si.quad(lambda x: f(x) / (eps - x), 0.0, top, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    im = -math.pi * f(eps) if eps > 0 else 0.0
    return pv + 1j * im


@pytest.mark.parametrize("l", [0, 1, 2])
@pytest.mark.parametrize("b", [0.25, 0.833])
@pytest.mark.parametrize("eps", [-1.3, -0.1, 0.05, 0.7, 2.0, 4.5])
def test_level_shift_matches_quadrature(l, b, eps):
    a = 0.186
    ref = _shift_by_quadrature(eps, a, b, l)
    got = complex(o.level_shift(np.array([eps]), a, b, l)[0])
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


def test_level_shift_width_relation_and_continuity():
    a, b, l = 0.1, 0.4, 1
    eps = np.linspace(0.01, 5, 50)
    F = o.level_shift(eps, a, b, l)
    np.testing.assert_allclose(-2 * F.imag, o.width(eps, a, b, l), rtol=1e-14)
    # real part is continuous through threshold: P_l(0) = -Gamma(l+1/2) b^-(l+1/2)
    F0 = o.level_shift(np.array([-1e-9, 0.0, 1e-9]), a, b, 0)
    np.testing.assert_allclose(F0.real, a / (2 * math.pi) * -math.sqrt(math.pi / b), rtol=1e-4)


# --------------------------------------------------------------- matrix properties
@pytest.fixture(scope="module")
def small_model():
    return w.ci2d_model(7, extra_terms=True)


def test_a_is_complex_symmetric_not_hermitian(small_model):
    A = o.a_matrix(small_model, 3.1).toarray()
    assert np.abs(A - A.T).max() <= 1e-14  # symmetric up to the summation order of terms
    assert np.abs(A - A.conj().T).max() > 1e-3


def test_anti_hermitian_part_is_open_channel_projector(small_model):
    E = 3.1
    A = o.a_matrix(small_model, E).toarray()
    anti = (A - A.conj().T) / 2j
    ref = np.zeros_like(anti)
    for nu in o.open_levels(small_model, E):
        for mu in range(o.n_partial_waves(small_model)):
            p = o.phi(small_model, E, nu, mu)
            ref += np.pi * np.outer(p, p)
    np.testing.assert_allclose(anti, ref, atol=1e-13)


@pytest.mark.parametrize("eps_i", [0.3, 1.7, 2.9])
def test_flux_conservation(small_model, eps_i):
    vi = [0, 0]
    E = o.total_energy(small_model, eps_i, vi)
    nmu = o.n_partial_waves(small_model)
    for mu_i in range(nmu):
        psi = o.solve(small_model, E, o.phi(small_model, E, vi, mu_i))
        t_ii = o.t_amplitude(small_model, E, vi, mu_i, psi)
        total = sum(abs(o.t_amplitude(small_model, E, vf, mf, psi)) ** 2
                    for vf in o.open_levels(small_model, E) for mf in range(nmu))
        assert total == pytest.approx(-t_ii.imag / math.pi, rel=1e-10)


def test_solve_residual_and_sparse_dense_agree():
    m = w.ci2d_model(12)
    E = o.total_energy(m, 2.2, [0, 0])
    rhs = o.phi(m, E, [0, 0], 0)
    x_dense = o.solve(m, E, rhs, dense_limit=10 ** 9)
    x_sparse = o.solve(m, E, rhs, dense_limit=0)
    assert o.relative_residual(m, E, x_dense, rhs) < 1e-13
    np.testing.assert_allclose(x_sparse, x_dense, rtol=1e-10, atol=1e-14)


# ------------------------------------------------------------- special-case limits
def test_diagonal_model_closed_form():
    m = w.ci2d_model(6)
    m["terms"] = [t for t in m["terms"] if not any(t["pow"])]  # keep E_d only
    eps_i, vi = 1.3, [1, 2]
    E = o.total_energy(m, eps_i, vi)
    en_v = float(o.level_energies(m)[o.flat_index(m, vi)])
    nmu = o.n_partial_waves(m)
    sig_ref = 0.0
    for ch in m["channels"]:
        d = ch["d"]
        e_d = [t["coef"] for t in m["terms"] if t["d"] == d][0]
        f = math.sqrt(ch["a"] * eps_i ** (ch["l"] + 0.5) * math.exp(-ch["b"] * eps_i) / (2 * math.pi))
        g = complex(o.level_shift(np.array([eps_i]), ch["a"], ch["b"], ch["l"])[0])
        t_ref = f * f / (E - en_v - e_d - g)
        psi = o.solve(m, E, o.phi(m, E, vi, ch["mu"]))
        assert o.t_amplitude(m, E, vi, ch["mu"], psi) == pytest.approx(t_ref, rel=1e-12)
        sig_ref += abs(t_ref) ** 2
        # flux identity holds algebraically: Im(1/(x - g)) = Im g / |x-g|^2, -Im g = pi f^2
        assert abs(t_ref) ** 2 == pytest.approx(-t_ref.imag / math.pi, rel=1e-12)
    sig, _ = o.cross_sections(m, [eps_i], [vi], [vi])
    assert sig[0, 0, 0] == pytest.approx(2 * math.pi ** 3 / eps_i * sig_ref, rel=1e-12)
    assert nmu == 2


def _dense_1d(omega, n, e_d, kappa, gamma, ch, E):
    """Directly built dense 1D matrix E - H for one state and one mode."""
    A = np.zeros((n, n), dtype=complex)
    for k in range(n):
        ek = omega * (k + 0.5)
        A[k, k] = E - ek - e_d - o.level_shift(np.array([E - ek]), ch["a"], ch["b"], ch["l"])[0]
    q = o.q_matrix(n)
    A -= kappa * q + gamma * (q @ q)
    return A


def test_decoupled_limit_factorises_into_1d_problems():
    m = w.ci2d_model(9)
    m["terms"] = [t for t in m["terms"] if t["pow"][1] == 0 and t["d"] == t["dp"]]
    ng, nu = m["modes"][0]["n"], m["modes"][1]["n"]
    wg, wu = m["modes"][0]["omega"], m["modes"][1]["omega"]
    vi = [0, 0]
    E = o.total_energy(m, 2.4, vi)
    for ch in m["channels"]:
        d = ch["d"]
        psi = o.solve(m, E, o.phi(m, E, vi, ch["mu"])).reshape(2, ng, nu)
        coef = {tuple(t["pow"]): t["coef"] for t in m["terms"] if t["d"] == d}
        for ku in range(nu):
            Eu = E - wu * (ku + 0.5)
            A1 = _dense_1d(wg, ng, coef[(0, 0)], coef[(1, 0)], coef[(2, 0)], ch, Eu)
            rhs = np.zeros(ng)
            if ku == 0:
                rhs[0] = o.coupling_amplitude(E - o.level_energies(m)[0], ch["a"], ch["b"], ch["l"])
            x1 = np.linalg.solve(A1, rhs)
            np.testing.assert_allclose(psi[d, :, ku], x1, rtol=1e-11, atol=1e-15)
        assert np.abs(psi[1 - d]).max() == 0.0


def test_eels_integrates_to_sum_of_cross_sections():
    m = w.ci2d_model(5)
    vf = o.open_levels(m, o.total_energy(m, 1.5, [0, 0]))
    sig = np.abs(np.random.default_rng(1).normal(size=(3, len(vf))))
    de = np.arange(-0.2, 3.0, 0.0005)
    S = o.eels(m, [1.0, 1.2, 1.5], [0, 0], vf, sig, de)
    np.testing.assert_allclose(S.sum(axis=1) * 0.0005, sig.sum(axis=1), rtol=1e-6)


def test_eels_single_line_width_and_position():
    """Eq. 2Dsp with a Gaussian of 10 meV FWHM: a single line of unit cross section sits at the
    energy loss E_vf - E_vi, peaks at 2 sqrt(ln 2 / pi) / FWHM (unit area) and falls to half of
    that 5 meV either side."""
    m = w.ci2d_model(5)
    wg = m["modes"][0]["omega"]
    fwhm = 0.010
    peak = 2.0 * math.sqrt(math.log(2.0) / math.pi) / fwhm
    for vf, loss in (([0, 0], 0.0), ([1, 0], wg)):
        de = np.array([loss - 0.005, loss, loss + 0.005, loss - 0.02])
        S = o.eels(m, [1.0], [0, 0], [vf], np.ones((1, 1)), de)[0]
        assert S[1] == pytest.approx(peak, rel=1e-12)
        assert S[0] == pytest.approx(0.5 * peak, rel=1e-12)
        assert S[2] == pytest.approx(0.5 * peak, rel=1e-12)
        assert S[3] == pytest.approx(peak * 2.0 ** (-16), rel=1e-9)  # 2 FWHM away: 2^-(2*2)^2


HARTREE_EV = 27.211386245988  # CODATA 2018


def _one_channel_model(e_d, a, b, l):
    """One discrete state, one vibrational function, one partial wave: A is the 1 x 1 matrix
    E - E_0 - e_d - F(E - E_0)."""
    return {"n_states": 1, "modes": [{"name": "x", "omega": 0.2, "n": 1}],
            "terms": [{"d": 0, "dp": 0, "coef": e_d, "pow": [0]}],
            "channels": [{"d": 0, "mu": 0, "a": a, "b": b, "l": l}]}


@pytest.mark.parametrize("e_d,a,b", [(1.0, 0.1, 0.5), (2.45, 0.186, 0.833)])
def test_cross_section_at_resonance_is_the_unitarity_limit(e_d, a, b):
    m = _one_channel_model(e_d, a, b, 0)
    re_a = lambda e: e - e_d - o.level_shift(np.array([e]), a, b, 0)[0].real
    eps_r = so.brentq(re_a, 0.05, 6.0, xtol=1e-15, rtol=1e-15)
    E = o.total_energy(m, eps_r, [0])
    psi = o.solve(m, E, o.phi(m, E, [0], 0))
    t = o.t_amplitude(m, E, [0], 0, psi)
    assert abs(t - (-1j / math.pi)) <= 1e-12
    sig, _ = o.cross_sections(m, [eps_r], [[0]], [[0]])
    k2 = 2.0 * eps_r / HARTREE_EV          # eps_i = k^2 / 2 in hartree
    sigma_bohr2 = sig[0, 0, 0] * HARTREE_EV  # the raw value takes eps_i in eV
    assert sigma_bohr2 == pytest.approx(4.0 * math.pi / k2, rel=1e-12)


def test_one_channel_amplitude_is_unitary_at_every_energy():
    m = _one_channel_model(1.0, 0.1, 0.5, 0)
    for eps_i in (0.05, 0.4, 0.99, 1.7, 3.5):
        E = o.total_energy(m, eps_i, [0])
        t = o.t_amplitude(m, E, [0], 0, o.solve(m, E, o.phi(m, E, [0], 0)))
        assert abs(1.0 - 2j * math.pi * t) == pytest.approx(1.0, abs=1e-13)
        sig, _ = o.cross_sections(m, [eps_i], [[0]], [[0]])
        assert sig[0, 0, 0] * HARTREE_EV <= 4.0 * math.pi / (2.0 * eps_i / HARTREE_EV) * (1 + 1e-12)


# ---------------------------------------------------------------------- gradient
def test_adjoint_gradient_matches_finite_differences():
    m = w.ci2d_model(5, extra_terms=True)
    eps = [1.1, 2.3]
    vi = [0, 0]
    vf = [[0, 0], [1, 0], [0, 1]]
    target = np.full((len(eps), len(vf)), 0.5)
    nt = len(m["terms"])
    thetas = [0, 1, 3, nt - 1, nt - 2, nt + 0, nt + 1, nt + 3]
    g_adj = o.loss_gradient_adjoint(m, eps, vi, vf, target, thetas)
    g_fd = o.loss_gradient_fd(m, eps, vi, vf, target, thetas, h=1e-6)
    np.testing.assert_allclose(g_adj, g_fd, rtol=2e-6, atol=1e-9 * np.abs(g_fd).max())


# -------------------------------------------------------------- paper parameters
def test_ecd86_parameters_match_table1():
    with open(os.path.join(GOLDEN, "ecd86_table1.json")) as fh:
        g = json.load(fh)["values"]
    m = w.ecd86_model(4, 4)
    assert m["modes"][0]["omega"] == g["omega_g"] and m["modes"][1]["omega"] == g["omega_u"]
    coef = {(t["d"], t["dp"], tuple(t["pow"])): t["coef"] for t in m["terms"]}
    assert coef[(0, 0, (0, 0))] == g["E1"] and coef[(1, 1, (0, 0))] == g["E2"]
    assert coef[(0, 0, (1, 0))] == g["kappa1"] and coef[(1, 1, (1, 0))] == g["kappa2"]
    assert coef[(0, 1, (0, 1))] == g["lambda"]
    ch = {c["d"]: c for c in m["channels"]}
    assert (ch[0]["a"], ch[0]["b"], ch[0]["l"]) == (g["a1"], g["b1"], g["l1"])
    assert (ch[1]["a"], ch[1]["b"], ch[1]["l"]) == (g["a2"], g["b2"], g["l2"])


# ------------------------------------------------------ preconditioner identities
def test_ecd86_preconditioner_identities():
    """Sec. III.B numerical testing, ECD86 paragraph: M^{dg} and M^{gu} hold only the diagonal of
    A, and M^{du}, M^{d}, M^{u} coincide (no q_u terms on the diagonal of U, and the
    inter-state coupling lambda q_u has no part diagonal in n_u)."""
    m = w.ecd86_model(6, 7)
    E = 3.3
    A = o.a_matrix(m, E)
    diag = sp_diag(A)
    span = {"dg": 0x4, "gu": 0x1, "du": 0x2, "d": 0x6, "g": 0x5, "u": 0x3}
    B = {k: o.block_diagonal(m, E, v).toarray() for k, v in span.items()}
    np.testing.assert_array_equal(B["dg"], diag)
    np.testing.assert_array_equal(B["gu"], diag)
    np.testing.assert_array_equal(B["du"], B["d"])
    np.testing.assert_array_equal(B["du"], B["u"])
    assert np.abs(B["g"] - B["du"]).max() > 0.1  # M^g holds the lambda coupling


def sp_diag(A):
    return np.diag(A.diagonal())


def test_block_labels_sizes():
    m = w.ci2d_model(5)
    for span, size in [(0x1, 2), (0x5, 10), (0x3, 10), (0x6, 25), (0x7, 50), (0x0, 1)]:
        lab = o.block_labels(m, span)
        _, counts = np.unique(lab, return_counts=True)
        assert set(counts) == {size}
