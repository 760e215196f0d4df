"""Pins of the oracle's generalized coupling V^mu_{d eps}(q) = f_d^mu(eps) P(q) (Sec. II.C).

The level-shift operator becomes the sandwich sum of Eq. FE, F_dd' = sum_mu P_dmu F[f_d f_d'] P_d'mu,
and Phi carries P(q)|v>.  Each pin rests on something other than the oracle's own code:

* the transform of a product of two channel amplitudes equals principal-value quadrature of
  its defining integral (Eq. IntF);
* with the unit polynomial the operator is the diagonal one of Sec. II.B (pinned separately),
  and a constant polynomial s acts as the width factor s^2;
* one mode with P = 1 + lambda q: the entries of P F P written out by hand from the ladder
  action of q (Sec. III), including the truncated last row; two states with P_1 = q_u, P_2 = 1:
  the off-diagonal block is q g, not g q (the operator order Eq. FE prescribes);
* A is complex symmetric and its anti-Hermitian part is exactly pi sum_{nu open, mu}
  Phi^{nu mu} Phi^{nu mu T} (Eq. F_gen with the i eta prescription), flux is conserved;
* the structure statement of Sec. III.C for the generalized model: every block choice of the
  preconditioners differs, except that M^{du} and M^u coincide;
* Table II's values are those of the generalized-model generator (golden file);
* the adjoint gradient with respect to coupling-polynomial coefficients matches central
  differences of the loss.
"""

import copy
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si

from oracle import vibronic as o
import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pair_by_quadrature(eps, ca, cb):
    """PV int_0^inf f_a(x) f_b(x) / (eps - x) dx - i pi f_a f_b(eps), f_c = sqrt(Gamma_c / 2 pi)."""

    def f(x):
        ga = ca["a"] * x ** (ca["l"] + 0.5) * math.exp(-ca["b"] * x)
        gb = cb["a"] * x ** (cb["l"] + 0.5) * math.exp(-cb["b"] * x)
        return math.sqrt(ga * gb) / (2.0 * math.pi)

    top = 120.0 / (ca["b"] + cb["b"]) + 10.0 * (ca["l"] + 1)
    if eps > 0:
        pv = -si.quad(f, 0.0, top, weight="cauchy", wvar=eps, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    else:
        pv = si.quad(lambda x: f(x) / (eps - x), 0.0, top, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    return pv - 1j * math.pi * (f(eps) if eps > 0 else 0.0)


@pytest.mark.parametrize("mu", [0, 1])
@pytest.mark.parametrize("eps", [-1.1, -0.05, 0.2, 1.3, 3.7])
def test_pair_transform_matches_quadrature(mu, eps):
    chans = [c for c in w.gen_ecd_model(3, 3)["channels"] if c["mu"] == mu]
    ca, cb = chans
    got = complex(o.pair_level_shift(np.array([eps]), ca, cb)[0])
    ref = _pair_by_quadrature(eps, ca, cb)
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


def test_pair_transform_of_a_channel_with_itself_is_its_level_shift():
    c = w.gen_ecd_model(3, 3)["channels"][2]
    eps = np.linspace(-2.0, 5.0, 29)
    np.testing.assert_allclose(o.pair_level_shift(eps, c, c), o.level_shift(eps, c["a"], c["b"], c["l"]),
                               rtol=1e-15, atol=1e-17)


def _diagonal_reference(m, E):
    """E - E_nu - U - diag(F) with the diagonal level shift of Sec. II.B (separately pinned)."""
    ns = m["n_states"]
    en = np.tile(o.level_energies(m), ns)
    return np.diag(E - en - o.continuum_diagonal(m, E)) - o.coupling_matrix(m).toarray()


def test_unit_polynomial_gives_the_diagonal_operator():
    m = w.ci2d_model(6)
    E = 3.05
    mu = copy.deepcopy(m)
    for c in mu["channels"]:
        c["terms"] = [{"coef": 1.0, "pow": [0, 0]}]
    np.testing.assert_allclose(o.a_matrix(mu, E).toarray(), _diagonal_reference(m, E), rtol=0, atol=1e-14)
    np.testing.assert_allclose(o.a_matrix(m, E).toarray(), _diagonal_reference(m, E), rtol=0, atol=1e-14)


def test_constant_polynomial_scales_the_width_quadratically():
    m = w.ci2d_model(5)
    E = 2.7
    s = 1.7
    ms, ma = copy.deepcopy(m), copy.deepcopy(m)
    ms["channels"][1]["terms"] = [{"coef": s, "pow": [0, 0]}]
    ma["channels"][1]["a"] *= s * s
    np.testing.assert_allclose(o.a_matrix(ms, E).toarray(), o.a_matrix(ma, E).toarray(), rtol=0, atol=1e-13)
    vi = [1, 0]
    np.testing.assert_allclose(o.phi(ms, E, vi, 1), o.phi(ma, E, vi, 1), rtol=1e-14)


def test_one_mode_sandwich_written_out_by_hand():
    """P = 1 + lam q on one mode: (P g P)(n, n') from <n|q|n+1> = sqrt((n+1)/2)."""
    n, lam = 7, 0.37
    ch = {"d": 0, "mu": 0, "a": 0.13, "b": 0.6, "l": 0,
          "terms": [{"coef": 1.0, "pow": [0]}, {"coef": lam, "pow": [1]}]}
    m = {"n_states": 1, "modes": [{"name": "x", "omega": 0.2, "n": n}], "terms": [], "channels": [ch]}
    E = 0.75
    g = o.level_shift(E - o.level_energies(m), ch["a"], ch["b"], 0)
    F = o.continuum_operator(m, E).toarray()
    s = lambda k: math.sqrt((k + 1) / 2.0)  # noqa: E731  <k|q|k+1>
    ref = np.zeros((n, n), dtype=complex)
    for k in range(n):
        ref[k, k] = g[k] + lam ** 2 * ((s(k - 1) ** 2 * g[k - 1] if k > 0 else 0) + (s(k) ** 2 * g[k + 1] if k + 1 < n else 0))
        if k + 1 < n:
            ref[k, k + 1] = ref[k + 1, k] = lam * s(k) * (g[k] + g[k + 1])
        if k + 2 < n:
            ref[k, k + 2] = ref[k + 2, k] = lam ** 2 * s(k) * s(k + 1) * g[k + 1]
    np.testing.assert_allclose(F, ref, rtol=1e-14, atol=1e-16)


def test_off_diagonal_block_keeps_the_operator_order():
    """P_1 = q, P_2 = 1 on one mode: F_12 = q g_12 (entries g_12 at the column index), F_21 = g_12 q."""
    n = 6
    c1 = {"d": 0, "mu": 0, "a": 0.1, "b": 0.5, "l": 0, "terms": [{"coef": 1.0, "pow": [1]}]}
    c2 = {"d": 1, "mu": 0, "a": 0.2, "b": 0.9, "l": 0}
    m = {"n_states": 2, "modes": [{"name": "x", "omega": 0.3, "n": n}], "terms": [], "channels": [c1, c2]}
    E = 1.4
    g12 = o.pair_level_shift(E - o.level_energies(m), c1, c2)
    F = o.continuum_operator(m, E).toarray()
    F12, F21 = F[:n, n:], F[n:, :n]
    for k in range(n - 1):
        s = math.sqrt((k + 1) / 2.0)
        assert F12[k, k + 1] == pytest.approx(s * g12[k + 1], rel=1e-14)
        assert F12[k + 1, k] == pytest.approx(s * g12[k], rel=1e-14)
    np.testing.assert_array_equal(F21, F12.T)
    assert np.abs(F12 - F12.T).max() > 1e-3  # the block itself is not symmetric


@pytest.fixture(scope="module")
def gen_small():
    return w.gen_ecd_model(7, 6)


def test_generalized_a_is_complex_symmetric(gen_small):
    A = o.a_matrix(gen_small, 3.4).toarray()
    assert np.abs(A - A.T).max() <= 1e-14
    assert np.abs(A - A.conj().T).max() > 1e-3


@pytest.mark.parametrize("E", [1.2, 3.4])
def test_generalized_anti_hermitian_part_is_open_channel_projector(gen_small, E):
    A = o.a_matrix(gen_small, E).toarray()
    anti = (A - A.conj().T) / 2j
    ref = np.zeros_like(anti)
    for nu in o.open_levels(gen_small, E):
        for mu in range(o.n_partial_waves(gen_small)):
            p = o.phi(gen_small, E, nu, mu)
            ref += np.pi * np.outer(p, p)
    assert np.abs(ref).max() > 1e-3
    np.testing.assert_allclose(anti, ref, atol=1e-13)


@pytest.mark.parametrize("eps_i", [0.4, 2.2, 3.9])
def test_generalized_flux_conservation(gen_small, eps_i):
    vi = [0, 0]
    E = o.total_energy(gen_small, eps_i, vi)
    nmu = o.n_partial_waves(gen_small)
    for mu_i in range(nmu):
        psi = o.solve(gen_small, E, o.phi(gen_small, E, vi, mu_i))
        t_ii = o.t_amplitude(gen_small, E, vi, mu_i, psi)
        total = sum(abs(o.t_amplitude(gen_small, E, vf, mf, psi)) ** 2
                    for vf in o.open_levels(gen_small, E) for mf in range(nmu))
        assert total == pytest.approx(-t_ii.imag / math.pi, rel=1e-10)


def test_generalized_phi_is_amplitude_times_polynomial_column(gen_small):
    """Phi^{v e} = f_1^e (1 + lam_1 q_g)|v> in state 1 and f_2^e q_u|v> in state 2 (Sec. II.C)."""
    m = gen_small
    E, v = 3.0, [2, 3]
    ng, nu = m["modes"][0]["n"], m["modes"][1]["n"]
    ev = o.level_energies(m)[o.flat_index(m, v)]
    c1, c2 = m["channels"][0], m["channels"][1]
    f1 = o.coupling_amplitude(E - ev, c1["a"], c1["b"], c1["l"])
    f2 = o.coupling_amplitude(E - ev, c2["a"], c2["b"], c2["l"])
    ref = np.zeros((2, ng, nu))
    ref[0, 2, 3] = f1
    ref[0, 1, 3] = f1 * 0.2 * math.sqrt(2 / 2.0)  # lam_1 <1|q_g|2>
    ref[0, 3, 3] = f1 * 0.2 * math.sqrt(3 / 2.0)  # lam_1 <3|q_g|2>
    ref[1, 2, 2] = f2 * math.sqrt(3 / 2.0)  # <2|q_u|3>
    ref[1, 2, 4] = f2 * math.sqrt(4 / 2.0)  # <4|q_u|3>
    np.testing.assert_allclose(o.phi(m, E, v, 0), ref.ravel(), rtol=1e-14, atol=1e-17)


def test_generalized_preconditioner_blocks_follow_the_paper():
    """Sec. III.C, generalized-model paragraph: all choices of diagonal blocks are distinct for
    this richer A, except that M^{du} and M^u coincide (every inter-state entry changes n_u)."""
    m = w.gen_ecd_model(6, 7)
    E = 3.3
    span = {"dg": 0x4, "gu": 0x1, "du": 0x2, "d": 0x6, "g": 0x5, "u": 0x3}
    B = {k: o.block_diagonal(m, E, v).toarray() for k, v in span.items()}
    np.testing.assert_array_equal(B["du"], B["u"])
    keys = ["dg", "gu", "du", "d", "g"]
    for i, a in enumerate(keys):
        for b in keys[i + 1:]:
            assert np.abs(B[a] - B[b]).max() > 1e-6, (a, b)


def test_generalized_parameters_match_table2():
    with open(os.path.join(GOLDEN, "gen_ecd_table2.json")) as fh:
        g = json.load(fh)["values"]
    m = w.gen_ecd_model(4, 4)
    ch = {(c["d"], c["mu"]): c for c in m["channels"]}
    for d in (1, 2):
        for mu, name in ((0, "e"), (1, "o")):
            c = ch[(d - 1, mu)]
            assert (c["a"], c["b"], c["l"]) == (g[f"a{d}{name}"], g[f"b{d}{name}"], g[f"l{d}{name}"])
    # V = [[f_1^e (1 + lambda_1 q_g), f_1^o q_u], [f_2^e q_u, f_2^o (1 + lambda_2 q_g)]]
    poly = lambda c: sorted((tuple(t["pow"]), t["coef"]) for t in c["terms"])  # noqa: E731
    assert poly(ch[(0, 0)]) == [((0, 0), 1.0), ((1, 0), g["lambda1"])]
    assert poly(ch[(1, 1)]) == [((0, 0), 1.0), ((1, 0), g["lambda2"])]
    assert poly(ch[(1, 0)]) == poly(ch[(0, 1)]) == [((0, 1), 1.0)]


def test_generalized_adjoint_gradient_matches_finite_differences():
    m = w.gen_ecd_model(5, 5)
    eps = [1.4, 3.1]
    vi = [0, 0]
    vf = [[0, 0], [1, 0], [0, 1]]
    target = np.full((len(eps), len(vf)), 0.05)
    nt, nc = len(m["terms"]), len(m["channels"])
    # E_1, lambda, a, b, lambda_1, the q_u coefficient of (d=2, e) alone, lambda_2
    thetas = [0, 4, nt + 0, nt + 3, nt + 2 * nc + 1, nt + 2 * nc + 2, nt + 2 * nc + 5]
    assert o.get_parameter(m, thetas[4]) == 0.2 and o.get_parameter(m, thetas[6]) == 0.1
    # each coefficient is a parameter of its own channel (no term shared between channels)
    m2 = o.with_parameter(m, thetas[5], 1.5)
    assert m2["channels"][1]["terms"][0]["coef"] == 1.5 and m2["channels"][2]["terms"][0]["coef"] == 1.0
    g_adj = o.loss_gradient_adjoint(m, eps, vi, vf, target, thetas)
    g_fd = o.loss_gradient_fd(m, eps, vi, vf, target, thetas, h=1e-6)
    np.testing.assert_allclose(g_adj, g_fd, rtol=2e-6, atol=1e-9 * np.abs(g_fd).max())
