"""CPU oracle for the vibronic-continuum linear systems (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import this module.  The CUDA path never calls it
and shares no code with it.

Everything here is the plain definition, in complex128 with NumPy/SciPy:

* per-mode truncated oscillator matrices (Sec. III, ladder action of q_g and q_u;
  Eq. H0harm for E_nu),
* the level-shift factor F[f](eps) (Eq. IntF with the widths of Sec. II.B), written in
  closed form through Dawson's function and the scaled complementary error function,
* the matrix A = E - H_ef = E - H_0 - U - F in the product basis (Eqs. H_ef, Amatrix),
  assembled as Kronecker products (state index slowest, last mode fastest); F is the
  operator of Eq. F_gen, diagonal for the q-independent couplings of Sec. II.B and the
  sandwich sum P F[f f'] P' of Eq. FE for the q-dependent couplings of Sec. II.C,
* the right-hand side Phi (Sec. II.D), the solve (Eq. Ax=b) by direct LU,
* T-matrix and cross section (Eqs. Td, crs, crs2), the 2D EELS sum (Eq. 2Dsp),
* the gradient of a cross-section loss by a dense-LU adjoint.

Readings of the paper taken here (the CUDA path takes the same ones):

* powers q^k are products of the truncated matrices (PqP)^k, the "successive
  multiplications" of Sec. III;
* f_d^mu(eps) = sqrt(Gamma_d^mu(eps) / 2 pi) is real and non-negative, and zero for
  eps <= 0 (closed channel);
* energies in eV; sigma is reported raw as 2 pi^3 |T|^2 / eps_i with eps_i in eV;
* a q-dependent coupling V^mu_{d eps}(q) = f_d^mu(eps) P(q) is separable (Sec. II.C) and its
  polynomial P(q) is a sum of products of truncated q matrices, like U; the channels of one
  partial wave share l, so that F[f f'] has the closed form of one channel;
* the EELS resolution function is a unit-area Gaussian of FWHM 10 meV.

Parity status: every function here is pinned by tests under ``tests/`` against
closed forms, quadrature, invariants or brute force (see the test module docstrings).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as sps

EELS_FWHM = 0.010  # eV, resolution of the spectrometer (Eq. 2Dsp)


# ----------------------------------------------------------------------------------------
# One-mode pieces (Sec. III; Eq. H0harm)
# ----------------------------------------------------------------------------------------
def q_matrix(n: int) -> np.ndarray:
    """Truncated coordinate operator: <k|q|k+1> = <k+1|q|k> = sqrt((k+1)/2) (Sec. III)."""
    q = np.zeros((n, n))
    k = np.arange(n - 1)
    q[k, k + 1] = np.sqrt((k + 1) / 2.0)
    q[k + 1, k] = q[k, k + 1]
    return q


def q_power(n: int, k: int) -> np.ndarray:
    """(PqP)^k: the k-th power of the truncated q matrix."""
    return np.linalg.matrix_power(q_matrix(n), k)


def mode_energies(omega: float, n: int) -> np.ndarray:
    """Harmonic levels omega (k + 1/2), k = 0..n-1 (Eq. H0harm)."""
    return omega * (np.arange(n) + 0.5)


def level_energies(model: dict) -> np.ndarray:
    """E_nu = sum_m omega_m (n_m + 1/2) over the product basis, last mode fastest."""
    e = np.zeros(1)
    for m in model["modes"]:
        e = (e[:, None] + mode_energies(m["omega"], m["n"])[None, :]).ravel()
    return e


def basis_shape(model: dict):
    return tuple(m["n"] for m in model["modes"])


def flat_index(model: dict, nu) -> int:
    """Position of the multi-index nu in the product basis (last mode fastest)."""
    return int(np.ravel_multi_index(tuple(nu), basis_shape(model)))


# ----------------------------------------------------------------------------------------
# Level shift (Eq. IntF, widths of Sec. II.B)
# ----------------------------------------------------------------------------------------
def width(eps, a: float, b: float, l: int):
    """Gamma(eps) = a eps^(l+1/2) exp(-b eps) for eps > 0, zero otherwise (Sec. II.B)."""
    eps = np.asarray(eps, dtype=np.float64)
    out = np.zeros_like(eps)
    pos = eps > 0
    out[pos] = a * eps[pos] ** (l + 0.5) * np.exp(-b * eps[pos])
    return out


def coupling_amplitude(eps, a: float, b: float, l: int):
    """f(eps) = sqrt(Gamma(eps)/(2 pi)), real, non-negative (Sec. II.C)."""
    return np.sqrt(width(eps, a, b, l) / (2.0 * np.pi))


def level_shift(eps, a: float, b: float, l: int):
    """F[Gamma/2pi](eps) = PV int f(x)/(eps-x) dx - i pi f(eps), f = Gamma/(2 pi) (Eq. IntF).

    With P_l(eps) = PV int_0^inf x^(l+1/2) e^(-bx) / (eps - x) dx the closed form is
      P_l = -Gamma(l+1/2) b^-(l+1/2) + eps P_(l-1),
      eps P_(-1) = 2 sqrt(pi eps) D(sqrt(b eps))          for eps > 0,
                 = pi sqrt(|eps|) erfcx(sqrt(b |eps|))     for eps < 0,
                 = 0                                       for eps = 0,
    where D is Dawson's function.  (Substituting x = t^2 turns P_(-1) into the Hilbert
    transform of a Gaussian for eps > 0 and into a Lorentzian-Gaussian integral for
    eps < 0.)  The imaginary part is -pi f(eps), so Gamma = -2 Im F (Sec. II.B).
    """
    eps = np.asarray(eps, dtype=np.float64)
    ae = np.abs(eps)
    eps_pm1 = np.where(
        eps > 0,
        2.0 * np.sqrt(np.pi * ae) * sps.dawsn(np.sqrt(b * ae)),
        np.pi * np.sqrt(ae) * sps.erfcx(np.sqrt(b * ae)),
    )
    eps_pm1 = np.where(eps == 0, 0.0, eps_pm1)
    p = -math.gamma(0.5) / math.sqrt(b) + eps_pm1  # P_0
    for k in range(1, l + 1):
        p = -math.gamma(k + 0.5) / b ** (k + 0.5) + eps * p
    re = a / (2.0 * np.pi) * p
    im = -np.pi * width(eps, a, b, l) / (2.0 * np.pi)
    return re + 1j * im


# ----------------------------------------------------------------------------------------
# The matrix A = E - H_ef (Eqs. H_ef, U, Amatrix)
# ----------------------------------------------------------------------------------------
def _kron_all(mats):
    out = sp.csr_matrix(np.ones((1, 1)))
    for m in mats:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


def lowering_matrix(n: int) -> np.ndarray:
    """Truncated annihilation operator of one oscillator: a|k> = sqrt(k)|k-1>."""
    a = np.zeros((n, n))
    k = np.arange(1, n)
    a[k - 1, k] = np.sqrt(k)
    return a


def ladder_matrix(n: int, j: int, k: int) -> np.ndarray:
    """(a^+)^j a^k as the product of truncated matrices (normal order: a^k acts first)."""
    a = lowering_matrix(n)
    return np.linalg.matrix_power(a.T, j) @ np.linalg.matrix_power(a, k)


def term_matrix(model: dict, pows, raises=None, lowers=None) -> sp.csr_matrix:
    """prod_m O_m on the vibrational product basis (Kronecker product), with O_m = q_m^(pow_m), or
    the ladder monomial (a_m^+)^raise_m a_m^lower_m when the term gives one for mode m."""
    mats = []
    for i, (m, k) in enumerate(zip(model["modes"], pows)):
        j = int(raises[i]) if raises else 0
        l = int(lowers[i]) if lowers else 0
        mats.append(ladder_matrix(m["n"], j, l) if (j or l) else q_power(m["n"], int(k)))
    return _kron_all(mats)


def term_operator(model: dict, t: dict) -> sp.csr_matrix:
    """The operator T of one term of U (coefficient excluded)."""
    return term_matrix(model, t["pow"], t.get("raise"), t.get("lower"))


def coupling_matrix(model: dict) -> sp.csr_matrix:
    """U (Eq. H_d / Eq. U) as a real symmetric sparse matrix over (d, nu).

    A term adds coef T to block (d, dp) and coef T^T to block (dp, d); on a diagonal block it
    adds the symmetric part coef (T + T^T) / 2 (T itself for powers of q, which are symmetric).
    Ladder monomials make T non-symmetric: they serve couplings written in circular (polar)
    oscillator quanta, where q_x +- i q_y = a_-+ + a_+-^+ have real matrix elements."""
    ns = model["n_states"]
    nv = int(np.prod(basis_shape(model)))
    blocks = [[sp.csr_matrix((nv, nv)) for _ in range(ns)] for _ in range(ns)]
    for t in model["terms"]:
        m = t["coef"] * term_operator(model, t)
        if t["d"] != t["dp"]:
            blocks[t["d"]][t["dp"]] = blocks[t["d"]][t["dp"]] + m
            blocks[t["dp"]][t["d"]] = blocks[t["dp"]][t["d"]] + m.T
        else:
            blocks[t["d"]][t["d"]] = blocks[t["d"]][t["d"]] + 0.5 * (m + m.T)
    return sp.bmat(blocks, format="csr")


def check_channels(model: dict):
    """A state couples to a partial wave at most once, and the channels of one partial wave
    share the exponent l (the closed form of F[f_c f_c'] in ``pair_level_shift`` needs it)."""
    seen, l_of = set(), {}
    for c in model["channels"]:
        if (c["d"], c["mu"]) in seen:
            raise ValueError("a state couples to a partial wave at most once")
        seen.add((c["d"], c["mu"]))
        if l_of.setdefault(c["mu"], c["l"]) != c["l"]:
            raise ValueError("the channels of one partial wave must share l")


def has_q_dependent_coupling(model: dict) -> bool:
    """True for the generalized coupling (Sec. II.C): some partial wave couples to two states
    or through a polynomial in q."""
    mus = [c["mu"] for c in model["channels"]]
    return len(set(mus)) != len(mus) or any(c.get("terms") for c in model["channels"])


def channel_polynomial(model: dict, c: int) -> sp.csr_matrix:
    """P_c(q) of the coupling V^mu_{d eps}(q) = f_d^mu(eps) P_c(q) (Sec. II.C, separable in eps
    and q): the sum of coef * prod_m q_m^pow over the channel's "terms", or the identity when it
    lists none (the q-independent coupling of Sec. II.B).  Real symmetric, N_nu x N_nu."""
    ch = model["channels"][c]
    nv = int(np.prod(basis_shape(model)))
    if not ch.get("terms"):
        return sp.identity(nv, format="csr")
    P = sp.csr_matrix((nv, nv))
    for t in ch["terms"]:
        P = P + t["coef"] * term_matrix(model, t["pow"])
    return P.tocsr()


def pair_level_shift(eps, ca: dict, cb: dict):
    """F[f_a f_b](eps) for two channels of one partial wave (Eq. FE, transform of Eq. IntF).

    With Gamma_c = a_c eps^(l+1/2) exp(-b_c eps) and f_c = sqrt(Gamma_c / 2 pi), the product is
    f_a f_b = (sqrt(a_a a_b) / 2 pi) eps^(l+1/2) exp(-(b_a + b_b) eps / 2): the one-channel
    form with a = sqrt(a_a a_b), b = (b_a + b_b) / 2, so ``level_shift`` applies (equal l)."""
    if ca["l"] != cb["l"]:
        raise ValueError("the channels of one partial wave must share l")
    return level_shift(eps, math.sqrt(ca["a"] * cb["a"]), 0.5 * (ca["b"] + cb["b"]), ca["l"])


def continuum_operator(model: dict, E: float) -> sp.csr_matrix:
    """The level-shift operator F(E - H_0) over alpha = (d, nu), complex128 (Eq. FE).

    For every partial wave mu and every ordered pair (c, c') of its channels, block (d_c, d_c')
    receives P_c diag(F[f_c f_c'](E - E_nu)) P_c'.  The factors keep this order: F is a function
    of E - H_0, which does not commute with q.  With q-independent couplings and one state per
    partial wave this is diag(F[Gamma_d / 2 pi](E - E_nu)) on the diagonal blocks (Sec. II.B)."""
    check_channels(model)
    ns = model["n_states"]
    nv = int(np.prod(basis_shape(model)))
    en = level_energies(model)
    chans = model["channels"]
    P = [channel_polynomial(model, c) for c in range(len(chans))]
    blocks = [[sp.csr_matrix((nv, nv), dtype=np.complex128) for _ in range(ns)] for _ in range(ns)]
    for c, ca in enumerate(chans):
        for cp, cb in enumerate(chans):
            if ca["mu"] != cb["mu"]:
                continue
            g = sp.diags(pair_level_shift(E - en, ca, cb))
            blocks[ca["d"]][cb["d"]] = blocks[ca["d"]][cb["d"]] + P[c] @ g @ P[cp]
    return sp.bmat(blocks, format="csr")


def continuum_diagonal(model: dict, E: float) -> np.ndarray:
    """Diagonal of F(E - H_0) for q-independent couplings with one state per partial wave
    (Sec. II.B): sum over the channels of state d of F[Gamma/2pi](E - E_nu)."""
    check_channels(model)
    if has_q_dependent_coupling(model):
        raise ValueError("F(E - H_0) is not diagonal for this coupling; use continuum_operator")
    ns = model["n_states"]
    en = level_energies(model)
    out = np.zeros((ns, en.size), dtype=np.complex128)
    for c in model["channels"]:
        out[c["d"]] += level_shift(E - en, c["a"], c["b"], c["l"])
    return out.ravel()


def a_matrix(model: dict, E: float) -> sp.csr_matrix:
    """A = E - H_0 - U - F(E - H_0) over alpha = (d, nu) (Eq. Amatrix), complex128."""
    ns = model["n_states"]
    en = np.tile(level_energies(model), ns)
    A = sp.diags((E - en).astype(np.complex128)) - coupling_matrix(model) - continuum_operator(model, E)
    return A.tocsr().astype(np.complex128)


# ----------------------------------------------------------------------------------------
# Right-hand sides, solve, observables (Eqs. Ax=b, Td, crs, crs2, 2Dsp)
# ----------------------------------------------------------------------------------------
def n_partial_waves(model: dict) -> int:
    return max(c["mu"] for c in model["channels"]) + 1


def phi(model: dict, E: float, v, mu: int) -> np.ndarray:
    """Phi^{v mu}_{d,nu} = <nu| V^mu_{d eps}(q) |v> with eps = E - E_v (Sec. II.D).

    With V^mu_{d eps} = f_d^mu(eps) P_c(q) (Sec. II.C) this is f_d^mu(E - E_v) times column v of
    P_c in the block of state d, summed over the channels c of mu; for q-independent couplings
    it is f_d^mu(E - E_v) on the single entry (d, v)."""
    ns = model["n_states"]
    nv = int(np.prod(basis_shape(model)))
    out = np.zeros(ns * nv)
    iv = flat_index(model, v)
    ev = float(level_energies(model)[iv])
    for k, c in enumerate(model["channels"]):
        if c["mu"] != mu:
            continue
        f = coupling_amplitude(E - ev, c["a"], c["b"], c["l"])
        if c.get("terms"):
            col = channel_polynomial(model, k)[:, iv].toarray().ravel()
            out[c["d"] * nv:(c["d"] + 1) * nv] += f * col
        else:
            out[c["d"] * nv + iv] += f
    return out


def total_energy(model: dict, eps_i: float, vi) -> float:
    """E = eps_i + E_vi (Eq. Econserv)."""
    return float(eps_i + level_energies(model)[flat_index(model, vi)])


def solve(model: dict, E: float, rhs: np.ndarray, dense_limit: int = 6000) -> np.ndarray:
    """psi = A^-1 rhs by direct LU (dense up to ``dense_limit`` unknowns, else sparse)."""
    A = a_matrix(model, E)
    if A.shape[0] <= dense_limit:
        return sla.lu_solve(sla.lu_factor(A.toarray()), rhs.astype(np.complex128))
    return spla.splu(A.tocsc()).solve(rhs.astype(np.complex128))


def solve_many(model: dict, E: float, rhss, dense_limit: int = 6000):
    """One LU factorisation, several right-hand sides (columns of the result)."""
    A = a_matrix(model, E)
    R = np.stack([np.asarray(r, dtype=np.complex128) for r in rhss], axis=1)
    if A.shape[0] <= dense_limit:
        return sla.lu_solve(sla.lu_factor(A.toarray()), R)
    return spla.splu(A.tocsc()).solve(R)


def relative_residual(model: dict, E: float, psi: np.ndarray, rhs: np.ndarray) -> float:
    """||rhs - A psi|| / ||rhs|| in complex128 (the stopping quantity of Sec. III)."""
    A = a_matrix(model, E)
    return float(np.linalg.norm(rhs - A @ psi) / np.linalg.norm(rhs))


def t_amplitude(model: dict, E: float, vf, mu_f: int, psi: np.ndarray) -> complex:
    """T_{mu_f v_f <- mu_i v_i} = <Phi^{v_f mu_f} | Psi> with real Phi (Eq. crs2)."""
    return complex(phi(model, E, vf, mu_f) @ psi)


def cross_section(eps_i: float, t_values) -> float:
    """sigma = 2 pi^3 / eps_i * sum |T|^2 over the listed (mu_i, mu_f) amplitudes (Eq. crs)."""
    t = np.asarray(t_values)
    return float(2.0 * np.pi ** 3 / eps_i * np.sum(np.abs(t) ** 2))


def cross_sections(model: dict, eps, vi_list, vf_list, dense_limit: int = 6000):
    """sigma[e, i, f] for incident energies eps, initial states vi_list, final vf_list.

    Sums over mu_i and mu_f (Eq. crs).  Also returns psi[e][i][mu_i] (flat vectors)."""
    nmu = n_partial_waves(model)
    sig = np.zeros((len(eps), len(vi_list), len(vf_list)))
    psis = []
    for e, ei in enumerate(eps):
        row = []
        for i, vi in enumerate(vi_list):
            E = total_energy(model, ei, vi)
            rhs = [phi(model, E, vi, mu) for mu in range(nmu)]
            ps = solve_many(model, E, rhs, dense_limit)
            row.append([ps[:, k] for k in range(nmu)])
            for f, vf in enumerate(vf_list):
                ts = [t_amplitude(model, E, vf, muf, ps[:, mi]) for mi in range(nmu) for muf in range(nmu)]
                sig[e, i, f] = cross_section(ei, ts)
        psis.append(row)
    return sig, psis


def open_levels(model: dict, E: float):
    """Multi-indices nu with E_nu < E (open final channels, eps_f > 0)."""
    en = level_energies(model)
    idx = np.nonzero(en < E)[0]
    return [list(np.unravel_index(int(k), basis_shape(model))) for k in idx]


def eels(model: dict, eps, vi, vf_list, sigma_ef: np.ndarray, de_grid, fwhm: float = EELS_FWHM):
    """S(eps_i, d_eps) = sum_f sigma_f(eps_i) rho(d_eps - (E_vf - E_vi)) (Eq. 2Dsp).

    rho is a unit-area Gaussian with the given FWHM.  sigma_ef[e, f]."""
    en = level_energies(model)
    e_vi = en[flat_index(model, vi)]
    shifts = np.array([en[flat_index(model, vf)] - e_vi for vf in vf_list])
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    de = np.asarray(de_grid, dtype=np.float64)
    rho = np.exp(-0.5 * ((de[None, :] - shifts[:, None]) / s) ** 2) / (s * math.sqrt(2.0 * math.pi))
    return np.asarray(sigma_ef) @ rho


# ----------------------------------------------------------------------------------------
# Gradient of L = sum (sigma - target)^2 by the dense-LU adjoint
# ----------------------------------------------------------------------------------------
def with_parameter(model: dict, theta: int, value: float) -> dict:
    """Copy of the model with parameter theta replaced.

    theta < n_terms: coefficient of term theta; n_terms <= theta < n_terms + 2 n_channels:
    channel c = (theta - n_terms) // 2, its ``a`` (even) or ``b`` (odd); beyond: the
    coefficients of the channels' coupling polynomials, channel by channel in listed order."""
    import copy

    m = copy.deepcopy(model)
    nt, nc = len(m["terms"]), len(m["channels"])
    if theta < nt:
        m["terms"][theta]["coef"] = value
    elif theta < nt + 2 * nc:
        c, which = divmod(theta - nt, 2)
        m["channels"][c]["ab"[which]] = value
    else:
        c, t = _poly_term(m, theta - nt - 2 * nc)
        m["channels"][c]["terms"][t]["coef"] = value
    return m


def _poly_term(model: dict, k: int):
    for c, ch in enumerate(model["channels"]):
        n = len(ch.get("terms") or [])
        if k < n:
            return c, k
        k -= n
    raise IndexError("parameter index beyond the coupling-polynomial terms")


def get_parameter(model: dict, theta: int) -> float:
    nt, nc = len(model["terms"]), len(model["channels"])
    if theta < nt:
        return float(model["terms"][theta]["coef"])
    if theta < nt + 2 * nc:
        c, which = divmod(theta - nt, 2)
        return float(model["channels"][c]["ab"[which]])
    c, t = _poly_term(model, theta - nt - 2 * nc)
    return float(model["channels"][c]["terms"][t]["coef"])


def loss(model: dict, eps, vi, vf_list, target) -> float:
    sig, _ = cross_sections(model, eps, [vi], vf_list)
    return float(np.sum((sig[:, 0, :] - target) ** 2))


def loss_gradient_fd(model: dict, eps, vi, vf_list, target, thetas, h: float = 1e-6):
    """Central finite differences of the loss with step h."""
    g = np.zeros(len(thetas))
    for k, th in enumerate(thetas):
        p0 = get_parameter(model, th)
        lp = loss(with_parameter(model, th, p0 + h), eps, vi, vf_list, target)
        lm = loss(with_parameter(model, th, p0 - h), eps, vi, vf_list, target)
        g[k] = (lp - lm) / (2.0 * h)
    return g


def loss_gradient_adjoint(model: dict, eps, vi, vf_list, target, thetas):
    """dL/dtheta by the adjoint of A psi = Phi with dense LU.

    T = Phi_f^T A^-1 Phi_i, so dT = dPhi_f^T psi + lambda_f^T dPhi_i - lambda_f^T dA psi
    with lambda_f = A^-T Phi_f = A^-1 Phi_f (A is complex symmetric).  dA/dtheta is
    obtained here by central differences of the assembled matrix in the parameter
    (A is linear in the term coefficients and in a, so the difference is exact for
    those up to rounding)."""
    nmu = n_partial_waves(model)
    grads = np.zeros(len(thetas))
    sig, _ = cross_sections(model, eps, [vi], vf_list)
    for e, ei in enumerate(eps):
        E = total_energy(model, ei, vi)
        A = a_matrix(model, E).toarray()
        lu = sla.lu_factor(A)
        phis_i = [phi(model, E, vi, mu) for mu in range(nmu)]
        psis = [sla.lu_solve(lu, p.astype(complex)) for p in phis_i]
        phis_f = [[phi(model, E, vf, mu) for mu in range(nmu)] for vf in vf_list]
        lams = [[sla.lu_solve(lu, p.astype(complex)) for p in row] for row in phis_f]
        for k, th in enumerate(thetas):
            p0 = get_parameter(model, th)
            hh = 1e-5 * max(1.0, abs(p0))
            mp, mm = with_parameter(model, th, p0 + hh), with_parameter(model, th, p0 - hh)
            dA = (a_matrix(mp, E).toarray() - a_matrix(mm, E).toarray()) / (2 * hh)
            dphi_i = [(phi(mp, E, vi, mu) - phi(mm, E, vi, mu)) / (2 * hh) for mu in range(nmu)]
            dphi_f = [[(phi(mp, E, vf, mu) - phi(mm, E, vf, mu)) / (2 * hh) for mu in range(nmu)] for vf in vf_list]
            tot = 0.0
            for f in range(len(vf_list)):
                w = 2.0 * (sig[e, 0, f] - target[e, f]) * 2.0 * np.pi ** 3 / ei
                for mi in range(nmu):
                    for mf in range(nmu):
                        T = phis_f[f][mf] @ psis[mi]
                        dT = dphi_f[f][mf] @ psis[mi] + lams[f][mf] @ dphi_i[mi] - lams[f][mf] @ (dA @ psis[mi])
                        tot += w * 2.0 * np.real(np.conj(T) * dT)
            grads[k] += tot
    return grads


# ----------------------------------------------------------------------------------------
# Block-diagonal preconditioners (Sec. III.B)
# ----------------------------------------------------------------------------------------
def block_labels(model: dict, span: int) -> np.ndarray:
    """Block label of every compound index alpha = (d, nu) for a preconditioner whose blocks
    span the indices in ``span`` (bit 0: state d, bit 1+m: mode m).  Two entries of A belong
    to the same block when all indices NOT spanned agree (Sec. III.B: the block-diagonal
    section of A)."""
    ns = model["n_states"]
    shape = (ns,) + basis_shape(model)
    grids = np.indices(shape).reshape(len(shape), -1)
    fixed = [k for k in range(len(shape)) if not (span >> k) & 1]
    if not fixed:
        return np.zeros(grids.shape[1], dtype=np.int64)
    sub = grids[fixed]
    dims = [shape[k] for k in fixed]
    return np.ravel_multi_index(tuple(sub), dims)


def block_diagonal(model: dict, E: float, span: int) -> sp.csr_matrix:
    """M = the entries of A whose row and column lie in the same block (Sec. III.B)."""
    A = a_matrix(model, E).tocoo()
    lab = block_labels(model, span)
    keep = lab[A.row] == lab[A.col]
    return sp.csr_matrix((A.data[keep], (A.row[keep], A.col[keep])), shape=A.shape)


def precond_apply(model: dict, E: float, span: int, r: np.ndarray) -> np.ndarray:
    """z = M^-1 r by a direct solve with the block-diagonal section M of A."""
    M = block_diagonal(model, E, span)
    return spla.splu(M.tocsc()).solve(np.asarray(r, dtype=np.complex128))
