"""Pins of the oracle's polar (circular-quanta) bending basis (Sec. III.C, CO2 paragraph: the
two-dimensional bend expanded in eigenfunctions of the 2D isotropic oscillator in polar
coordinates) and of its ladder-operator terms, against facts fixed outside the oracle:

* truncated ladder matrices: <n-k+j|(a^+)^j a^k|n> = sqrt(n!/(n-k)!) sqrt((n-k+j)!/(n-k)!),
  a^+ a = diag(n), and the truncated a a^+ loses the top level;
* the polar eigenfunctions |n_+, n_-> (angular momentum l = n_+ - n_-, shell v = n_+ + n_-)
  are built from the Cartesian ones by the binomial expansion of
  (a_x^+ + i a_y^+)^n_+ (a_x^+ - i a_y^+)^n_- / sqrt(2^v n_+! n_-!); that map is unitary on
  every shell, and it carries q_x + i q_y and q_x - i q_y (built from powers of q in the
  Cartesian product basis) into a_- + a_+^+ and a_+ + a_-^+ (built from ladder monomials in the
  circular product basis);
* the 2D isotropic oscillator has levels omega (v + 1) with degeneracy v + 1, and isotropic
  couplings (functions of rho^2, up to rho^4) conserve l;
* the Renner-Teller bend block of the CO2-like model (states Pi_x, Pi_y, Cartesian bend) and
  the same block in the Pi_+-, circular basis are one operator: the matrices agree under
  the unitary map on every shell the truncation leaves complete, and the low-lying spectra
  agree; the circular form conserves K = Lambda + l.
"""

import math

import numpy as np
import pytest

from oracle import vibronic as o


def _binom(n, k):
    return math.comb(n, k)


def polar_to_cartesian(N):
    """U[(nx, ny), (np, nm)]: coefficient of |nx, ny> in |n_+, n_->, for every pair with
    np + nm = nx + ny <= N - 1 (complete shells of both N x N product bases); index of a pair
    (a, b) is a * N + b."""
    U = np.zeros((N * N, N * N), dtype=complex)
    for v in range(N):
        for npl in range(v + 1):
            nm = v - npl
            norm = 1.0 / math.sqrt(2.0 ** v * math.factorial(npl) * math.factorial(nm))
            for p in range(npl + 1):          # a_x^+ taken p times from the first factor
                for q in range(nm + 1):       # and q times from the second
                    nx = p + q
                    ny = v - nx
                    c = _binom(npl, p) * _binom(nm, q) * (1j) ** (npl - p) * (-1j) ** (nm - q)
                    U[nx * N + ny, npl * N + nm] += c * norm * math.sqrt(math.factorial(nx) * math.factorial(ny))
    return U


def _shell_index(N, vmax):
    """Indices (a * N + b) of the pairs with a + b <= vmax."""
    return np.array([a * N + b for a in range(N) for b in range(N) if a + b <= vmax])


def _bend(N, names):
    return {"n_states": 1, "modes": [{"name": names[0], "omega": 0.1, "n": N}, {"name": names[1], "omega": 0.1, "n": N}],
            "terms": [], "channels": [{"d": 0, "mu": 0, "a": 0.0, "b": 1.0, "l": 0}]}


# ------------------------------------------------------------------ ladder matrices
def test_ladder_matrix_elements():
    n = 9
    for j in range(4):
        for k in range(4):
            L = o.ladder_matrix(n, j, k)
            for m in range(n):
                for r in range(n):
                    ref = 0.0
                    if m >= k and r == m - k + j and r < n:
                        ref = math.sqrt(math.factorial(m) / math.factorial(m - k)) * \
                            math.sqrt(math.factorial(m - k + j) / math.factorial(m - k))
                    assert L[r, m] == pytest.approx(ref, abs=1e-12)
    np.testing.assert_allclose(o.ladder_matrix(n, 1, 1), np.diag(np.arange(n)), atol=1e-14)
    aad = o.lowering_matrix(n) @ o.lowering_matrix(n).T
    np.testing.assert_allclose(np.diag(aad)[:-1], np.arange(1, n), atol=1e-14)
    assert aad[n - 1, n - 1] == 0.0  # truncation: the top level has no a^+ partner


def test_polar_map_is_unitary_on_every_shell():
    N = 8
    U = polar_to_cartesian(N)
    idx = _shell_index(N, N - 1)
    Us = U[np.ix_(idx, idx)]
    np.testing.assert_allclose(Us.conj().T @ Us, np.eye(idx.size), atol=1e-12)


def test_circular_ladders_are_the_cartesian_complex_coordinates():
    N = 9
    U = polar_to_cartesian(N)
    cart = _bend(N, ("x", "y"))
    qx = o.term_matrix(cart, [1, 0]).toarray()
    qy = o.term_matrix(cart, [0, 1]).toarray()
    circ = _bend(N, ("+", "-"))
    w_plus = (o.term_matrix(circ, [0, 0], [0, 0], [0, 1]) + o.term_matrix(circ, [0, 0], [1, 0], [0, 0])).toarray()
    w_minus = (o.term_matrix(circ, [0, 0], [0, 0], [1, 0]) + o.term_matrix(circ, [0, 0], [0, 1], [0, 0])).toarray()
    rows = _shell_index(N, N - 2)   # q changes v by one: these rows stay inside complete shells
    cols = _shell_index(N, N - 1)
    for cart_op, circ_op in ((qx + 1j * qy, w_plus), (qx - 1j * qy, w_minus)):
        ref = (U.conj().T @ cart_op @ U)[np.ix_(rows, cols)]
        np.testing.assert_allclose(circ_op[np.ix_(rows, cols)], ref, atol=1e-12)


# ----------------------------------------------------------- the 2D isotropic oscillator
def _rho2_terms(coef, d=0):
    """coef rho^2 = coef (a_+ a_- + a_+^+ a_-^+ + n_+ + n_- + 1) as ladder terms on state d.
    (On a diagonal block a term adds its symmetric part, so a_+ a_- + h.c. needs coef.)"""
    return [{"d": d, "dp": d, "coef": 2 * coef, "pow": [0, 0], "raise": [0, 0], "lower": [1, 1]},
            {"d": d, "dp": d, "coef": coef, "pow": [0, 0], "raise": [1, 0], "lower": [1, 0]},
            {"d": d, "dp": d, "coef": coef, "pow": [0, 0], "raise": [0, 1], "lower": [0, 1]},
            {"d": d, "dp": d, "coef": coef, "pow": [0, 0]}]


def test_isotropic_oscillator_levels_and_degeneracy():
    N, om = 12, 0.083
    m = _bend(N, ("+", "-"))
    m["modes"][0]["omega"] = m["modes"][1]["omega"] = om
    E = o.level_energies(m).reshape(N, N)
    for v in range(N):
        shell = [E[a, v - a] for a in range(v + 1)]
        np.testing.assert_allclose(shell, om * (v + 1), atol=1e-14)  # v + 1 states at omega (v + 1)


def test_rho2_and_rho4_conserve_angular_momentum_and_match_cartesian():
    N = 10
    U = polar_to_cartesian(N)
    circ = _bend(N, ("+", "-"))
    circ["terms"] = _rho2_terms(1.0)
    R2 = o.coupling_matrix(circ).toarray()
    cart = _bend(N, ("x", "y"))
    R2c = (o.term_matrix(cart, [2, 0]) + o.term_matrix(cart, [0, 2])).toarray()
    rows = _shell_index(N, N - 3)
    cols = _shell_index(N, N - 1)
    np.testing.assert_allclose(R2[np.ix_(rows, cols)], (U.conj().T @ R2c @ U)[np.ix_(rows, cols)], atol=1e-12)
    ell = np.array([a - b for a in range(N) for b in range(N)])
    R4 = R2 @ R2  # a quartic isotropic coupling
    for M in (R2, R4):
        i, j = np.nonzero(np.abs(M) > 1e-13)
        assert i.size > 0 and np.all(ell[i] == ell[j])


# ------------------------------------------------------------- Renner-Teller bend block
def _rt_cartesian(N, gamma, c):
    """States Pi_x, Pi_y; bend x, y: gamma rho^2 + c (q_x^2 - q_y^2) on Pi_x, - c on Pi_y,
    2 c q_x q_y between them (the CO2-like model's bend block)."""
    m = {"n_states": 2, "modes": [{"name": "x", "omega": 0.083, "n": N}, {"name": "y", "omega": 0.083, "n": N}],
         "channels": [{"d": 0, "mu": 0, "a": 0.0, "b": 1.0, "l": 1}, {"d": 1, "mu": 1, "a": 0.0, "b": 1.0, "l": 1}],
         "terms": []}
    for d, sgn in ((0, 1.0), (1, -1.0)):
        m["terms"] += [{"d": d, "dp": d, "coef": gamma + sgn * c, "pow": [2, 0]},
                       {"d": d, "dp": d, "coef": gamma - sgn * c, "pow": [0, 2]}]
    m["terms"].append({"d": 0, "dp": 1, "coef": 2 * c, "pow": [1, 1]})
    return m


def _rt_circular(N, gamma, c):
    """States Pi_+, Pi_-; circular bend quanta +, -: gamma rho^2 on both, and
    <Pi_+|H|Pi_-> = c (q_x - i q_y)^2 = c (a_+ + a_-^+)^2 = c (a_+^2 + 2 a_+ a_-^+ + a_-^+2)."""
    m = {"n_states": 2, "modes": [{"name": "+", "omega": 0.083, "n": N}, {"name": "-", "omega": 0.083, "n": N}],
         "channels": [{"d": 0, "mu": 0, "a": 0.0, "b": 1.0, "l": 1}, {"d": 1, "mu": 1, "a": 0.0, "b": 1.0, "l": 1}],
         "terms": _rho2_terms(gamma, 0) + _rho2_terms(gamma, 1)}
    m["terms"] += [{"d": 0, "dp": 1, "coef": c, "pow": [0, 0], "raise": [0, 0], "lower": [2, 0]},
                   {"d": 0, "dp": 1, "coef": 2 * c, "pow": [0, 0], "raise": [0, 1], "lower": [1, 0]},
                   {"d": 0, "dp": 1, "coef": c, "pow": [0, 0], "raise": [0, 2], "lower": [0, 0]}]
    return m


def _hamiltonian(m):
    ns = m["n_states"]
    return np.diag(np.tile(o.level_energies(m), ns)) + o.coupling_matrix(m).toarray()


def test_renner_teller_block_is_the_same_operator_in_both_bases():
    N, gamma, c = 10, 0.031, -0.008
    Hc = _hamiltonian(_rt_cartesian(N, gamma, c))
    Hp = _hamiltonian(_rt_circular(N, gamma, c))
    U = polar_to_cartesian(N)
    # Pi_+- = (Pi_x +- i Pi_y) / sqrt 2 on the electronic index
    Ue = np.array([[1.0, 1.0], [1j, -1j]]) / math.sqrt(2.0)
    W = np.kron(Ue, U)
    nv = N * N
    rows = np.concatenate([_shell_index(N, N - 3) + d * nv for d in range(2)])
    cols = np.concatenate([_shell_index(N, N - 1) + d * nv for d in range(2)])
    np.testing.assert_allclose(Hp[np.ix_(rows, cols)], (W.conj().T @ Hc @ W)[np.ix_(rows, cols)], atol=1e-12)


def test_renner_teller_spectra_agree_and_k_is_conserved():
    N, gamma, c = 28, 0.031, -0.008
    ec = np.sort(np.linalg.eigvalsh(_hamiltonian(_rt_cartesian(N, gamma, c))))[:12]
    Hp = _hamiltonian(_rt_circular(N, gamma, c))
    assert np.abs(Hp - Hp.T).max() <= 1e-15  # real symmetric: A stays complex symmetric
    ep = np.sort(np.linalg.eigvalsh(Hp))[:12]
    np.testing.assert_allclose(ep, ec, atol=1e-9)
    nv = N * N
    ell = np.array([a - b for a in range(N) for b in range(N)])
    K = np.concatenate([ell + 1, ell - 1])  # Lambda = +1 for Pi_+, -1 for Pi_-
    i, j = np.nonzero(np.abs(Hp) > 1e-13)
    assert np.all(K[i] == K[j])
    assert nv == ell.size


def test_polar_co2_workload_is_complex_symmetric_and_conserves_k():
    import workloads as w

    m = w.co2_polar_model(basis=(3, 6, 6, 2))
    A = o.a_matrix(m, 3.5).toarray()
    assert np.abs(A - A.T).max() == 0.0
    shape = (3,) + tuple(md["n"] for md in m["modes"])
    idx = np.indices(shape).reshape(len(shape), -1)
    K = idx[2] - idx[3] + np.array([0, 1, -1])[idx[0]]  # l = n_+ - n_-, Lambda = 0, +1, -1
    i, j = np.nonzero(np.abs(A) > 1e-13)
    assert np.all(K[i] == K[j])
    # every coupling kind is present: Sigma-Pi, Pi_+ - Pi_-, and fourth-order bend terms
    deg = [sum(t.get("raise", [0] * 4)) + sum(t.get("lower", [0] * 4)) for t in m["terms"]]
    assert max(deg) == 4 and any(t["d"] == 1 and t["dp"] == 2 for t in m["terms"])
