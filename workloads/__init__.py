"""Seeded synthetic model descriptions shared by the oracle side and the CUDA side.

This module only draws random parameters and lays out grids; it holds none of the
method's arithmetic (no oscillator matrices, no level shift, no solve).  Both the
oracle (``oracle/``) and the GPU path (``paper_2307_13483_gb300``) read the plain
dictionaries it returns.

Model dictionary format (all energies in eV, Sec. II):

* ``n_states``  number of discrete anion states d (Sec. II.A, Eq. H_d).
* ``modes``     list of {"name", "omega", "n"}: harmonic frequency omega_m and the
                number of oscillator functions kept, n_m = 0..n-1 (Eq. H0harm, Sec. II.D).
* ``terms``     polynomial terms of the direct vibronic coupling U_{dd'}(q)
                (Eq. U): {"d", "dp", "coef", "pow"} means coef * prod_m q_m^pow[m] in
                block (d, dp).  Only d <= dp is listed; U is symmetric, so a term with
                d < dp also stands in block (dp, d).  The state energies E_d are the
                terms with all powers zero.
* ``channels``  discrete-state/continuum couplings with constant q-dependence
                (Sec. II.B): {"d", "mu", "a", "b", "l"} gives the width
                Gamma_d^mu(eps) = a * eps^(l+1/2) * exp(-b*eps) of state d into
                partial wave mu.  An optional "terms" list [{"coef", "pow"}] makes
                the coupling q-dependent, V^mu_{d eps}(q) = f_d^mu(eps) P(q) with
                P(q) = sum coef * prod_m q_m^pow[m] (Sec. II.C); a partial wave may
                then couple to several states, whose channels share l.
"""

from __future__ import annotations

import numpy as np

CI2D_SEED = 2307134830
CO2_SEED = 2307134833


def _u(rng, lo, hi):
    return float(rng.uniform(lo, hi))


def ci2d_model(n_basis: int = 40, seed: int = CI2D_SEED, extra_terms: bool = False) -> dict:
    """2-state, 2-mode conical-intersection model shaped like the ECD86 model (Eq. U).

    State d=0 is even and couples to the even partial wave mu=0; state d=1 is odd and
    couples to mu=1 (Sec. II.B).  Mode 0 is the totally symmetric q_g, mode 1 the
    coupling mode q_u.  Diagonal terms are even in q_u and off-diagonal terms odd in
    q_u, as the symmetry requires.

    Recipe: omega_g, omega_u ~ U(0.1, 0.3); E_d ~ U(2.0, 3.0); kappa_d q_g,
    gamma_{d,gg} q_g^2, gamma_{d,uu} q_u^2 and lambda q_u ~ U(-0.2, 0.2), with the
    quadratic coefficients clipped to >= -0.4 omega so every diabatic potential stays
    bound; widths Gamma_d = A_d sqrt(eps) exp(-eps/B_d), A_d ~ U(0.05, 0.2),
    B_d ~ U(1, 4) (so l = 0, b = 1/B_d).  With ``extra_terms`` the model also gets the
    cubic and bilinear terms used for the gradient workload, coefficients
    ~ U(-0.02, 0.02): kappa'_d q_g^3, gamma'_d q_g q_u^2 (diagonal) and
    lambda' q_g q_u, lambda'' q_u^3 (off-diagonal).
    """
    rng = np.random.default_rng(seed)
    wg = _u(rng, 0.1, 0.3)
    wu = _u(rng, 0.1, 0.3)
    terms = []
    for d in range(2):
        terms.append({"d": d, "dp": d, "coef": _u(rng, 2.0, 3.0), "pow": [0, 0]})
        terms.append({"d": d, "dp": d, "coef": _u(rng, -0.2, 0.2), "pow": [1, 0]})
        terms.append({"d": d, "dp": d, "coef": max(_u(rng, -0.2, 0.2), -0.4 * wg), "pow": [2, 0]})
        terms.append({"d": d, "dp": d, "coef": max(_u(rng, -0.2, 0.2), -0.4 * wu), "pow": [0, 2]})
    terms.append({"d": 0, "dp": 1, "coef": _u(rng, -0.2, 0.2), "pow": [0, 1]})
    channels = []
    for d in range(2):
        A = _u(rng, 0.05, 0.2)
        B = _u(rng, 1.0, 4.0)
        channels.append({"d": d, "mu": d, "a": A, "b": 1.0 / B, "l": 0})
    if extra_terms:
        for d in range(2):
            terms.append({"d": d, "dp": d, "coef": _u(rng, -0.02, 0.02), "pow": [3, 0]})
            terms.append({"d": d, "dp": d, "coef": _u(rng, -0.02, 0.02), "pow": [1, 2]})
        terms.append({"d": 0, "dp": 1, "coef": _u(rng, -0.02, 0.02), "pow": [1, 1]})
        terms.append({"d": 0, "dp": 1, "coef": _u(rng, -0.02, 0.02), "pow": [0, 3]})
    return {
        "name": f"ci2d-{n_basis}" + ("-x" if extra_terms else ""),
        "seed": seed,
        "n_states": 2,
        "modes": [{"name": "g", "omega": wg, "n": n_basis}, {"name": "u", "omega": wu, "n": n_basis}],
        "terms": terms,
        "channels": channels,
    }


def co2_like_model(basis=(30, 20, 20, 12), seed: int = CO2_SEED) -> dict:
    """3-state, 4-mode model shaped like the paper's CO2 model (Sec. III.B, CO2 paragraph).

    States: d=0 a Sigma virtual state (width with l=0), d=1,2 the two components Pi_x,
    Pi_y of a shape resonance (l=1); each couples to its own partial wave.  Modes:
    symmetric stretch s1, bend components bx, by, asymmetric stretch s3, with CO2's
    fundamentals as frequencies (0.172, 0.083, 0.083, 0.291 eV).  Couplings
    ~ U(-0.2, 0.2) eV: stretch linear/quadratic terms on the diagonals, an isotropic
    bend quadratic, Renner-Teller terms c (q_bx^2 - q_by^2) on Pi_x and -c on Pi_y,
    a bilinear Pi_x-Pi_y coupling 2c q_bx q_by, Sigma-Pi_x ~ q_bx and Sigma-Pi_y ~ q_by.
    Quadratic diagonal coefficients are clipped to >= -0.4 omega.  E_Sigma ~ U(1, 2),
    E_Pi ~ U(3, 4) eV; widths a ~ U(0.05, 0.2), b = 1/B with B ~ U(1, 4).
    """
    rng = np.random.default_rng(seed)
    om = [0.172, 0.083, 0.083, 0.291]
    modes = [{"name": nm, "omega": w, "n": int(n)} for nm, w, n in zip(("s1", "bx", "by", "s3"), om, basis)]
    terms = []

    def t(d, dp, c, p):
        terms.append({"d": d, "dp": dp, "coef": float(c), "pow": list(p)})

    e_sig = _u(rng, 1.0, 2.0)
    e_pi = _u(rng, 3.0, 4.0)
    k_sig, k_pi = _u(rng, -0.2, 0.2), _u(rng, -0.2, 0.2)
    g1_sig, g1_pi = max(_u(rng, -0.2, 0.2), -0.4 * om[0]), max(_u(rng, -0.2, 0.2), -0.4 * om[0])
    g3_sig, g3_pi = max(_u(rng, -0.2, 0.2), -0.4 * om[3]), max(_u(rng, -0.2, 0.2), -0.4 * om[3])
    gb_sig, gb_pi = max(_u(rng, -0.2, 0.2), -0.3 * om[1]), max(_u(rng, -0.2, 0.2), -0.3 * om[1])
    c_rt = float(np.clip(_u(rng, -0.2, 0.2), -0.1 * om[1], 0.1 * om[1]))
    lam_sp = _u(rng, -0.2, 0.2)
    t(0, 0, e_sig, (0, 0, 0, 0))
    t(0, 0, k_sig, (1, 0, 0, 0))
    t(0, 0, g1_sig, (2, 0, 0, 0))
    t(0, 0, g3_sig, (0, 0, 0, 2))
    t(0, 0, gb_sig, (0, 2, 0, 0))
    t(0, 0, gb_sig, (0, 0, 2, 0))
    for d, sgn in ((1, 1.0), (2, -1.0)):
        t(d, d, e_pi, (0, 0, 0, 0))
        t(d, d, k_pi, (1, 0, 0, 0))
        t(d, d, g1_pi, (2, 0, 0, 0))
        t(d, d, g3_pi, (0, 0, 0, 2))
        t(d, d, gb_pi + sgn * c_rt, (0, 2, 0, 0))
        t(d, d, gb_pi - sgn * c_rt, (0, 0, 2, 0))
    t(1, 2, 2.0 * c_rt, (0, 1, 1, 0))
    t(0, 1, lam_sp, (0, 1, 0, 0))
    t(0, 2, lam_sp, (0, 0, 1, 0))
    channels = [
        {"d": 0, "mu": 0, "a": _u(rng, 0.05, 0.2), "b": 1.0 / _u(rng, 1.0, 4.0), "l": 0},
    ]
    a_pi, b_pi = _u(rng, 0.05, 0.2), 1.0 / _u(rng, 1.0, 4.0)
    channels.append({"d": 1, "mu": 1, "a": a_pi, "b": b_pi, "l": 1})
    channels.append({"d": 2, "mu": 2, "a": a_pi, "b": b_pi, "l": 1})
    return {
        "name": "co2like-" + "x".join(str(n) for n in basis),
        "seed": seed,
        "n_states": 3,
        "modes": modes,
        "terms": terms,
        "channels": channels,
    }


def co2_polar_model(basis=(30, 20, 20, 12), seed: int = CO2_SEED) -> dict:
    """The CO2-like model with its bend in polar form (Sec. III.C, CO2 paragraph: the 2D bend in
    eigenfunctions of the 2D isotropic oscillator in polar coordinates, couplings up to fourth
    order).  The bend basis is the product of the circular quanta n_+, n_- (modes 1 and 2, both
    of frequency omega_b: the polar states with v = n_+ + n_-, l = n_+ - n_-), truncated at
    n_+-  < basis[1]; the electronic states are Sigma (d=0) and Pi_+, Pi_- (d=1, 2:
    (Pi_x +- i Pi_y)/sqrt 2), so every coupling has real ladder-operator coefficients.

    Recipe (seeded like ``co2_like_model``, couplings ~ U(-0.2, 0.2) eV): stretch linear and
    quadratic terms on each state; isotropic bend terms gamma rho^2 with
    rho^2 = a_+ a_- + a_+^+ a_-^+ + n_+ + n_- + 1; fourth-order isotropic bend terms
    c1 n_+ n_- + c2 ((a_+ a_-)^2 + h.c.) + c3 (a_+^+2 a_+^2 + a_-^+2 a_-^2) with c ~ U(-0.004, 0.004);
    the Renner-Teller coupling <Pi_+|H|Pi_-> = c (a_+ + a_-^+)^2; Sigma-Pi couplings
    <Sigma|H|Pi_+-> = lambda (a_-+ + a_+-^+) / sqrt 2.  All of them conserve K = Lambda + l."""
    rng = np.random.default_rng(seed + 7)
    om = [0.172, 0.083, 0.083, 0.291]
    modes = [{"name": nm, "omega": w, "n": int(n)} for nm, w, n in zip(("s1", "b+", "b-", "s3"), om, basis)]
    terms = []

    def t(d, dp, c, p=(0, 0, 0, 0), r=(0, 0, 0, 0), lo=(0, 0, 0, 0)):
        terms.append({"d": d, "dp": dp, "coef": float(c), "pow": list(p), "raise": list(r), "lower": list(lo)})

    def rho2(d, c):
        t(d, d, 2 * c, lo=(0, 1, 1, 0))          # a_+ a_- + h.c. (a diagonal block keeps the symmetric part)
        t(d, d, c, r=(0, 1, 0, 0), lo=(0, 1, 0, 0))
        t(d, d, c, r=(0, 0, 1, 0), lo=(0, 0, 1, 0))
        t(d, d, c)

    e_sig, e_pi = _u(rng, 1.0, 2.0), _u(rng, 3.0, 4.0)
    for d in range(3):
        t(d, d, e_sig if d == 0 else e_pi)
        t(d, d, _u(rng, -0.2, 0.2), p=(1, 0, 0, 0))
        t(d, d, max(_u(rng, -0.2, 0.2), -0.4 * om[0]), p=(2, 0, 0, 0))
        t(d, d, max(_u(rng, -0.2, 0.2), -0.4 * om[3]), p=(0, 0, 0, 2))
        rho2(d, max(_u(rng, -0.2, 0.2), -0.3 * om[1]))
        t(d, d, _u(rng, -0.004, 0.004), r=(0, 1, 1, 0), lo=(0, 1, 1, 0))
        t(d, d, 2 * _u(rng, -0.004, 0.004), lo=(0, 2, 2, 0))
        c3 = _u(rng, -0.004, 0.004)
        t(d, d, c3, r=(0, 2, 0, 0), lo=(0, 2, 0, 0))
        t(d, d, c3, r=(0, 0, 2, 0), lo=(0, 0, 2, 0))
    c_rt = float(np.clip(_u(rng, -0.2, 0.2), -0.1 * om[1], 0.1 * om[1]))
    t(1, 2, c_rt, lo=(0, 2, 0, 0))
    t(1, 2, 2 * c_rt, r=(0, 0, 1, 0), lo=(0, 1, 0, 0))
    t(1, 2, c_rt, r=(0, 0, 2, 0))
    lam = _u(rng, -0.2, 0.2) / np.sqrt(2.0)
    t(0, 1, lam, lo=(0, 0, 1, 0))
    t(0, 1, lam, r=(0, 1, 0, 0))
    t(0, 2, lam, lo=(0, 1, 0, 0))
    t(0, 2, lam, r=(0, 0, 1, 0))
    a_pi, b_pi = _u(rng, 0.05, 0.2), 1.0 / _u(rng, 1.0, 4.0)
    channels = [{"d": 0, "mu": 0, "a": _u(rng, 0.05, 0.2), "b": 1.0 / _u(rng, 1.0, 4.0), "l": 0},
                {"d": 1, "mu": 1, "a": a_pi, "b": b_pi, "l": 1},
                {"d": 2, "mu": 2, "a": a_pi, "b": b_pi, "l": 1}]
    return {"name": "co2polar-" + "x".join(str(n) for n in basis), "seed": seed + 7, "n_states": 3, "modes": modes,
            "terms": terms, "channels": channels}


def ecd86_model(n_g: int, n_u: int) -> dict:
    """The ECD86 pseudo-Jahn-Teller model with the parameter values of Table I.

    U = [[E1 + kappa1 q_g, lambda q_u], [lambda q_u, E2 + kappa2 q_g]] (Eq. U);
    Gamma_d = a_d eps^(l_d+1/2) exp(-b_d eps); d=1 couples to the even wave and d=2 to
    the odd wave (Sec. II.B).  Index d here is 0-based.
    """
    return {
        "name": f"ecd86-{n_g}x{n_u}",
        "seed": None,
        "n_states": 2,
        "modes": [{"name": "g", "omega": 0.258, "n": n_g}, {"name": "u", "omega": 0.091, "n": n_u}],
        "terms": [
            {"d": 0, "dp": 0, "coef": 2.45, "pow": [0, 0]},
            {"d": 1, "dp": 1, "coef": 2.85, "pow": [0, 0]},
            {"d": 0, "dp": 0, "coef": -0.212, "pow": [1, 0]},
            {"d": 1, "dp": 1, "coef": 0.254, "pow": [1, 0]},
            {"d": 0, "dp": 1, "coef": 0.318, "pow": [0, 1]},
        ],
        "channels": [
            {"d": 0, "mu": 0, "a": 0.086, "b": 0.833, "l": 2},
            {"d": 1, "mu": 1, "a": 0.186, "b": 0.375, "l": 1},
        ],
    }


def gen_ecd_model(n_g: int, n_u: int) -> dict:
    """The generalized model of Sec. II.C with the parameter values of Tables I and II.

    U is the ECD86 matrix of Table I; the coupling matrix is expanded to first order in q,
      V = [[f_1^e (1 + lambda_1 q_g), f_1^o q_u], [f_2^e q_u, f_2^o (1 + lambda_2 q_g)]]
    (rows d, columns mu = e, o), with 2 pi |f_d^mu|^2 = a eps^(l+1/2) exp(-b eps) from
    Table II.  Both partial waves couple to both states.  Index d here is 0-based.
    """
    m = ecd86_model(n_g, n_u)
    lam1, lam2 = 0.2, 0.1
    # every channel gets its own term list (its coefficients are parameters of their own)
    one_plus = lambda lam: [{"coef": 1.0, "pow": [0, 0]}, {"coef": lam, "pow": [1, 0]}]  # noqa: E731
    q_u = lambda: [{"coef": 1.0, "pow": [0, 1]}]  # noqa: E731
    m["name"] = f"gen-ecd-{n_g}x{n_u}"
    m["channels"] = [
        {"d": 0, "mu": 0, "a": 0.07, "b": 0.25, "l": 0, "terms": one_plus(lam1)},
        {"d": 1, "mu": 0, "a": 0.1, "b": 0.5, "l": 0, "terms": q_u()},
        {"d": 0, "mu": 1, "a": 0.186, "b": 0.375, "l": 1, "terms": q_u()},
        {"d": 1, "mu": 1, "a": 0.15, "b": 0.8, "l": 1, "terms": one_plus(lam2)},
    ]
    return m


def eps_grid(eps_max: float, n: int) -> np.ndarray:
    """Incident electron energies eps_k = eps_max * k / n, k = 1..n (zero excluded)."""
    return eps_max * np.arange(1, n + 1, dtype=np.float64) / n


def lowest_levels(model: dict, count: int) -> list:
    """The ``count`` oscillator multi-indices with the smallest sum of omega_m * n_m.

    Used to pick initial vibrational states; ties are broken by the multi-index order.
    """
    import itertools

    ranges = [range(min(m["n"], count)) for m in model["modes"]]
    cands = []
    for idx in itertools.product(*ranges):
        cands.append((sum(m["omega"] * k for m, k in zip(model["modes"], idx)), idx))
    cands.sort()
    return [list(c[1]) for c in cands[:count]]


# Workloads (sizes and seeds of the five configurations the benchmarks and tests use).
WORKLOADS = {
    "ci2d_single": dict(model=lambda: ci2d_model(40), eps=np.array([1.0]), vi=[[0, 0]]),
    "ci2d_batched": dict(model=lambda: ci2d_model(80), eps=eps_grid(3.0, 256), vi=[[0, 0]]),
    "co2_like": dict(model=lambda: co2_like_model(), eps=np.array([3.0]), vi=[[0, 0, 0, 0]]),
    "co2_polar": dict(model=lambda: co2_polar_model(), eps=np.array([3.0]), vi=[[0, 0, 0, 0]]),
    "ci2d_uneven": dict(model=lambda: ci2d_model(80), eps=eps_grid(4.0, 128), vi=None),
    "ci2d_adjoint": dict(model=lambda: ci2d_model(40, extra_terms=True), eps=eps_grid(3.0, 256), vi=[[0, 0]]),
}
