"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Sizes are chosen so that the oracle finishes in seconds while the kernels still see several
thread blocks and a ragged tail (N not a multiple of the block sizes).  Tolerances:
  * FP64 operator: relative 1e-13 (rounding of ~20 terms per entry);
  * FP32 operator: relative 2e-6 (single-precision rounding of the same sums);
  * solves: the true residual ||Phi - A psi|| / ||Phi|| computed by the oracle in complex128
    must meet the requested tolerance, and cross sections must agree with the LU solution
    to 1e-8 relative when the tolerance is 1e-10 (sigma ~ |T|^2 and the error of T is bounded
    by cond(A) * tol);
  * adjoint gradient: 1e-6 relative against the oracle's dense-LU adjoint.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as w  # noqa: E402
from oracle import vibronic as o  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vbk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2307_13483_gb300 as lib

    return lib


def rand_vectors(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


MODELS = {
    "ci2d_x": lambda: w.ci2d_model(9, extra_terms=True) | {"modes": [{"name": "g", "omega": 0.21, "n": 37},
                                                                     {"name": "u", "omega": 0.13, "n": 29}]},
    "ecd86": lambda: w.ecd86_model(11, 23),
    "co2_small": lambda: w.co2_like_model(basis=(5, 4, 4, 3)),
    "one_mode": lambda: {"n_states": 1, "modes": [{"name": "x", "omega": 0.2, "n": 300}],
                         "terms": [{"d": 0, "dp": 0, "coef": 1.1, "pow": [0]}, {"d": 0, "dp": 0, "coef": 0.15, "pow": [1]},
                                   {"d": 0, "dp": 0, "coef": 0.02, "pow": [3]}],
                         "channels": [{"d": 0, "mu": 0, "a": 0.1, "b": 0.5, "l": 2}]},
    "frozen_mode": lambda: w.ci2d_model(5) | {"modes": [{"name": "g", "omega": 0.25, "n": 33},
                                                        {"name": "u", "omega": 0.12, "n": 1}]},
}


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("variant", list(range(20)))  # VBK_MATVEC_NVARIANTS
def test_matvec_parity(vbk, name, precision, variant):
    """Every matvec kernel variant (direct / shared-memory-windowed, 1..8 systems per thread)."""
    desc = MODELS[name]()
    model = vbk.Model(desc)
    rng = np.random.default_rng(7)
    E = np.array([0.35, 2.6, 4.1])
    nvec = 3  # 9 systems: a ragged last group for every systems-per-thread count
    x = rand_vectors(rng, (E.size, nvec, model.N))
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
        for k in range(nvec):
            ref = A @ x[e, k]
            err = np.abs(y[e, k] - ref)
            assert err.max() <= tol * np.abs(ref).max() * 4, (name, e, k, err.max())
            assert np.linalg.norm(y[e, k] - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("span", [-1, 0, 0x1, 0x5, 0x3, 0x2, 0x4, 0x6, 0x7])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_precond_parity(vbk, span, precision):
    # 13 x 4 oscillator functions keep every chain bandwidth <= 16 (span 0x7 without the cubic terms)
    desc = w.ci2d_model(7, extra_terms=span != 0x7)
    desc["modes"][0]["n"], desc["modes"][1]["n"] = 13, 4
    model = vbk.Model(desc)
    rng = np.random.default_rng(11)
    E = np.array([1.2, 3.4])
    r = rand_vectors(rng, (E.size, 3, model.N))
    z = vbk.vbk_precond_apply(model, E, torch.tensor(r, device="cuda"), span,
                              precision=0 if precision == "fp64" else 1).cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 5e-5
    for e in range(E.size):
        for k in range(3):
            ref = r[e, k] if span < 0 else o.precond_apply(desc, E[e], span if span > 0 else 0, r[e, k])
            assert np.linalg.norm(z[e, k] - ref) <= tol * np.linalg.norm(ref), (span, e, k)


def test_preconditioner_identities_on_gpu(vbk):
    """ECD86: the factors of M^{dg}, M^{gu} give the Jacobi result and M^{du}, M^{d}, M^{u} agree
    (Sec. III.B numerical testing)."""
    desc = w.ecd86_model(6, 7)
    model = vbk.Model(desc)
    rng = np.random.default_rng(3)
    r = torch.tensor(rand_vectors(rng, (1, 2, model.N)), device="cuda")
    E = [3.3]
    z = {s: vbk.vbk_precond_apply(model, E, r, s).cpu().numpy() for s in (0, 0x4, 0x1, 0x2, 0x6, 0x3)}
    np.testing.assert_allclose(z[0x4], z[0], rtol=1e-13, atol=0)
    np.testing.assert_allclose(z[0x1], z[0], rtol=1e-13, atol=0)
    np.testing.assert_allclose(z[0x6], z[0x2], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(z[0x3], z[0x2], rtol=1e-12, atol=1e-300)


def _oracle_psi(desc, eps, vi):
    nmu = o.n_partial_waves(desc)
    out = np.zeros((len(eps), len(vi), nmu, o.a_matrix(desc, 1.0).shape[0]), dtype=complex)
    for e, ei in enumerate(eps):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, ei, v)
            ps = o.solve_many(desc, E, [o.phi(desc, E, v, mu) for mu in range(nmu)])
            out[e, i] = ps.T
    return out


SOLVERS = [
    ("gmres", "fp64", 0),
    ("gmres", "mixed", 0),
    ("gmres", "mixed", 0x5),
    ("gmres", "fp64", -1),
    ("cocg", "fp64", 0),
    ("cocg", "mixed", 0),
    ("cocg", "mixed", 0x5),
    ("cocg", "fp64", 0x1),
]


@pytest.mark.parametrize("name", ["ci2d_x", "ecd86", "co2_small", "one_mode", "frozen_mode"])
@pytest.mark.parametrize("span,resident", [(0, 1), (-1, 1), (0, 2), (0, 3), (-1, 3)])
def test_resident_paths_on_every_model_shape(vbk, name, span, resident):
    """The fused solves -- resident = 1: the whole refinement of each system in one thread block;
    resident = 3: one cluster of n_s thread blocks per system -- and the one-block inner solves
    (resident = 2) on 1 to 3 states, 1 to 4 modes, bilinear points with a second mode and a frozen
    mode, Jacobi or no preconditioner: true residuals by the oracle."""
    desc = MODELS[name]()
    model = vbk.Model(desc)
    eps = np.array([0.3, 1.1, 2.4, 3.3])
    vi = [[0] * len(desc["modes"])]
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=span, tol=1e-10, resident=resident,
                                max_iter=40000, max_refine=400)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    psi = psi.cpu().numpy()
    for e, ei in enumerate(eps):
        E = o.total_energy(desc, ei, vi[0])
        A = o.a_matrix(desc, E)
        for mu in range(model.n_mu):
            st = stats[e * model.n_mu + mu]
            rhs = o.phi(desc, E, vi[0], mu)
            if not np.any(rhs):
                assert st["status"] == "zero_rhs"
                continue
            assert st["status"] == "converged", (e, mu, st)
            res = np.linalg.norm(rhs - A @ psi[e, 0, mu]) / np.linalg.norm(rhs)
            assert res <= 1e-10 * 1.05, (e, mu, res, st)


@pytest.mark.parametrize("nb", [(12, 12), (40, 40), (64, 64), (80, 80), (5, 4, 8, 3)])
def test_fused_solve_quad_shapes(vbk, nb):
    """The fused one-block solve on models whose second-fastest mode has a multiple of 4 functions
    (its stencil loops take quads of elements): fewer quads than threads, a whole number of
    passes (64 x 64), a ragged last pass (80 x 80, the batched workload's size) and four modes
    with three states (the CO2-like model without its bilinear coupling).  True residuals and
    cross sections by the oracle."""
    if len(nb) == 2:
        desc = w.ci2d_model(nb[0])
        desc["modes"][1]["n"] = nb[1]
    else:
        desc = w.co2_like_model(basis=nb)
        desc["terms"] = [t for t in desc["terms"] if sum(1 for p in t["pow"] if p) <= 1]
    model = vbk.Model(desc)
    assert model.N == desc["n_states"] * int(np.prod([m["n"] for m in desc["modes"]]))
    eps = np.array([0.35, 1.6, 2.8])
    vi = [[0] * len(desc["modes"])]
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=0, tol=1e-10, resident=1,
                                max_iter=40000, max_refine=400)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    psi = psi.cpu().numpy()
    for e, ei in enumerate(eps):
        E = o.total_energy(desc, ei, vi[0])
        A = o.a_matrix(desc, E)
        for mu in range(model.n_mu):
            st = stats[e * model.n_mu + mu]
            rhs = o.phi(desc, E, vi[0], mu)
            if not np.any(rhs):
                assert st["status"] == "zero_rhs"
                continue
            assert st["status"] == "converged", (e, mu, st)
            res = np.linalg.norm(rhs - A @ psi[e, 0, mu]) / np.linalg.norm(rhs)
            assert res <= 1e-10 * 1.05, (e, mu, res, st)
    vf = o.open_levels(desc, o.total_energy(desc, eps[-1], vi[0]))[:8]
    sig = vbk.vbk_cross_sections(model, eps, vi, torch.tensor(psi, device="cuda"), vf).cpu().numpy()
    sig_ref, _ = o.cross_sections(desc, eps, vi, vf)
    big = np.abs(sig_ref) > 1e-6 * np.abs(sig_ref).max()
    assert (np.abs(sig - sig_ref)[big] / np.abs(sig_ref)[big]).max() <= 1e-8


@pytest.mark.parametrize("method,precision,span", SOLVERS)
def test_solve_parity(vbk, method, precision, span):
    desc = w.ci2d_model(14)
    desc["modes"][1]["n"] = 11  # N = 2 * 14 * 11 = 308
    model = vbk.Model(desc)
    eps = np.array([0.4, 1.3, 2.2, 2.9])
    vi = [[0, 0], [1, 0]]
    opts = vbk.vbk_default_opts(method=method, precision=precision, precond_span=span, tol=1e-10, restart=40,
                                max_iter=20000, max_refine=200)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    psi = psi.cpu().numpy()
    ref = _oracle_psi(desc, eps, vi)
    nmu = model.n_mu
    for e, ei in enumerate(eps):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, ei, v)
            for mu in range(nmu):
                st = stats[(e * len(vi) + i) * nmu + mu]
                assert st["status"] == "converged", st
                rhs = o.phi(desc, E, v, mu)
                res = o.relative_residual(desc, E, psi[e, i, mu], rhs)
                assert res <= 1e-10 * 1.05, (e, i, mu, res, st)
                assert abs(st["rel_residual"] - res) <= 1e-12 + 0.05 * res
    vf = o.open_levels(desc, o.total_energy(desc, eps[-1], vi[-1]))[:12]
    sig = vbk.vbk_cross_sections(model, eps, vi, torch.tensor(psi, device="cuda"), vf).cpu().numpy()
    sig_ref, _ = o.cross_sections(desc, eps, vi, vf)
    big = np.abs(sig_ref) > 1e-6 * np.abs(sig_ref).max()
    rel = np.abs(sig - sig_ref)[big] / np.abs(sig_ref)[big]
    assert rel.max() <= 1e-8, rel.max()


@pytest.mark.parametrize("method,precision", [("cocg", "mixed"), ("gmres", "mixed"), ("cocg", "fp64")])
@pytest.mark.parametrize("variant", list(range(20)))  # VBK_MATVEC_NVARIANTS
def test_solve_with_every_matvec_variant(vbk, method, precision, variant):
    """The grid-wide solve (resident = 0) with each matvec variant fixed for the Krylov operator
    and the FP64 residual: the variants' partial sums (dot products, residual norms: one slot per
    system and block or strip) and their system lists (converged systems retire) must serve the
    solver; true residuals by the oracle."""
    desc = w.ci2d_model(10)
    # N = 2 * 10 * 80 = 1600: rows of 80 entries, so that the streaming variants' FP64 plans take
    # shorter strips than their FP32 plans (different partial counts in one mixed solve)
    desc["modes"][1]["n"] = 80
    model = vbk.Model(desc)
    eps = np.array([0.4, 1.3, 2.2, 2.9])
    vi = [[0, 0], [1, 0]]
    opts = vbk.vbk_default_opts(method=method, precision=precision, precond_span=0, tol=1e-10, restart=40,
                                max_iter=20000, max_refine=200, resident=0, matvec_variant=variant)
    try:
        psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    except vbk.VbkError as err:
        if err.code == 1 and "variant not available" in str(err):
            pytest.skip("variant does not fit this model")
        raise
    psi = psi.cpu().numpy()
    for e, ei in enumerate(eps):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, ei, v)
            for mu in range(model.n_mu):
                st = stats[(e * len(vi) + i) * model.n_mu + mu]
                assert st["status"] == "converged", st
                res = o.relative_residual(desc, E, psi[e, i, mu], o.phi(desc, E, v, mu))
                assert res <= 1e-10 * 1.05, (e, i, mu, res, st)


def test_cross_sections_and_t_match_oracle_on_oracle_psi(vbk):
    """Readout alone: sigma and T from the oracle's own psi (Eqs. crs, crs2)."""
    desc = w.ci2d_model(8)
    model = vbk.Model(desc)
    eps = np.array([0.7, 2.5])
    vi = [[0, 0], [0, 1]]
    psi = _oracle_psi(desc, eps, vi)
    vf = [[0, 0], [1, 0], [0, 1], [2, 1], [7, 7]]
    sig, T = vbk.vbk_cross_sections(model, eps, vi, torch.tensor(psi, device="cuda"), vf, want_t=True)
    sig, T = sig.cpu().numpy(), T.cpu().numpy()
    sig_ref, _ = o.cross_sections(desc, eps, vi, vf)
    np.testing.assert_allclose(sig, sig_ref, rtol=1e-13, atol=1e-300)
    for e, ei in enumerate(eps):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, ei, v)
            for mi in range(2):
                for f, fv in enumerate(vf):
                    for mf in range(2):
                        t_ref = o.t_amplitude(desc, E, fv, mf, psi[e, i, mi])
                        assert abs(T[e, i, mi, f, mf] - t_ref) <= 1e-14 * max(1e-300, abs(t_ref)) + 1e-300


def test_flux_conservation_of_gpu_solutions(vbk):
    desc = w.ci2d_model(12, extra_terms=True)
    model = vbk.Model(desc)
    eps = np.array([0.5, 1.5, 2.5, 3.5])
    vi = [[0, 0]]
    opts = vbk.vbk_default_opts(method="gmres", precision="mixed", tol=1e-11, restart=48, max_refine=200)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    for e, ei in enumerate(eps):
        E = o.total_energy(desc, ei, vi[0])
        vf = o.open_levels(desc, E)
        psi_e = torch.tensor(psi[e:e + 1].cpu().numpy(), device="cuda")
        _, T = vbk.vbk_cross_sections(model, eps[e:e + 1], vi, psi_e, vf, want_t=True)
        T = T.cpu().numpy()[0, 0]  # [mu_i, f, mu_f]
        for mi in range(2):
            total = np.sum(np.abs(T[mi]) ** 2)
            t_ii = T[mi, vf.index([0, 0]), mi]
            assert total == pytest.approx(-t_ii.imag / math.pi, rel=1e-8)


def test_eels_matches_oracle(vbk):
    desc = w.ci2d_model(8)
    model = vbk.Model(desc)
    eps = np.array([1.0, 2.0])
    vi = [[0, 0]]
    vf = o.open_levels(desc, o.total_energy(desc, 2.0, vi[0]))
    rng = np.random.default_rng(5)
    sig = np.abs(rng.standard_normal((2, 1, len(vf))))
    de = np.arange(-0.1, 2.5, 0.001)
    S = vbk.vbk_eels(model, vi, vf, torch.tensor(sig, device="cuda"), de).cpu().numpy()
    for e in range(2):
        ref = o.eels(desc, eps[e:e + 1], vi[0], vf, sig[e:e + 1, 0], de)[0]
        np.testing.assert_allclose(S[e, 0], ref, rtol=1e-12, atol=1e-12 * ref.max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_gradient_matches_oracle(vbk, precision):
    desc = w.ci2d_model(5, extra_terms=True)
    model = vbk.Model(desc)
    eps = np.array([1.1, 2.3])
    vi = [[0, 0]]
    vf = [[0, 0], [1, 0], [0, 1]]
    target = np.full((2, 3), 0.5)
    nt = len(desc["terms"])
    thetas = list(range(nt)) + [nt, nt + 1, nt + 2, nt + 3]
    g_ref = o.loss_gradient_adjoint(desc, eps, vi[0], vf, target, thetas)
    opts = vbk.vbk_default_opts(method="gmres", precision=precision, tol=1e-12, restart=50, max_refine=100)
    psi, _ = vbk.vbk_solve(model, eps, vi, opts)
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf)
    dlds = 2.0 * (sig - torch.tensor(target[:, None, :], device="cuda"))
    g, stats = vbk.vbk_solve_adjoint(model, eps, vi, psi, vf, dlds, thetas, opts)
    assert all(s["status"] == "converged" for s in stats)
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-9 * np.abs(g_ref).max())


def test_autograd_function_matches_finite_differences(vbk):
    desc = w.ci2d_model(5, extra_terms=True)
    eps = np.array([1.1, 2.3])
    vi = [[0, 0]]
    vf = [[0, 0], [1, 0], [0, 1]]
    target = torch.full((2, 1, 3), 0.5, dtype=torch.float64, device="cuda")
    nt = len(desc["terms"])
    ids = [1, 4, nt - 1, nt, nt + 3]
    vals = torch.tensor([o.get_parameter(desc, k) for k in ids], dtype=torch.float64, requires_grad=True)
    opts = vbk.vbk_default_opts(method="gmres", precision="fp64", tol=1e-13, restart=50)
    sig = vbk.cross_sections_torch(vals, desc, ids, eps, vi, vf, opts)
    L = ((sig - target) ** 2).sum()
    L.backward()
    g_fd = o.loss_gradient_fd(desc, eps, vi[0], vf, target[:, 0].cpu().numpy(), ids, h=1e-6)
    np.testing.assert_allclose(vals.grad.numpy(), g_fd, rtol=2e-6, atol=1e-8 * np.abs(g_fd).max())


def test_edge_cases(vbk):
    desc = w.ci2d_model(6)
    model = vbk.Model(desc)
    # closed channel -> zero right-hand side (a = 0 for mu = 1)
    d2 = w.ci2d_model(6)
    d2["channels"][1]["a"] = 0.0
    m2 = vbk.Model(d2)
    psi, st = vbk.vbk_solve(m2, [1.0], [[0, 0]], vbk.vbk_default_opts(tol=1e-10))
    assert st[1]["status"] == "zero_rhs" and st[0]["status"] == "converged"
    assert float(psi[0, 0, 1].abs().max()) == 0.0
    # invalid arguments
    with pytest.raises(vbk.VbkError):
        vbk.vbk_solve(model, [-1.0], [[0, 0]])
    with pytest.raises(vbk.VbkError):
        vbk.vbk_solve(model, [1.0], [[6, 0]])
    with pytest.raises(vbk.VbkError):
        vbk.vbk_solve(model, [1.0], [[0, 0]], vbk.vbk_default_opts(restart=0))
    # iteration cap reported per system
    psi, st = vbk.vbk_solve(model, [2.0], [[0, 0]], vbk.vbk_default_opts(max_iter=1, max_refine=1, tol=1e-12),
                            check=False)
    assert all(s["status"] == "max_iter" for s in st)
    # maximum restart length and a single-iteration check interval
    psi, st = vbk.vbk_solve(model, [2.0], [[0, 0]], vbk.vbk_default_opts(restart=256, check_every=1, tol=1e-10))
    assert all(s["status"] == "converged" for s in st)
    with pytest.raises(vbk.VbkError):
        vbk.vbk_solve(model, [1.0], [[0, 0]], vbk.vbk_default_opts(inner_max_iter=-1))


def _zero_pivot_model():
    """Two states, binary-fraction parameters, no continuum on state 1: at eps_i = 1.125 eV from
    v_i = (0, 0) the diagonal entry of A at (d = 1, nu = (0, 1)) is E - E_nu - E_1 = 0 exactly
    (E = 1.3125, E_nu = 0.3125, E_1 = 1), a zero pivot of the point preconditioner and of the
    span-d blocks (lambda q_u couples the states only across n_u, so those blocks are diagonal).
    The entry lies in the symmetry sector of Phi ((0, even n_u) with (1, odd n_u)), so the
    Krylov iterates reach it."""
    return {"n_states": 2, "modes": [{"name": "g", "omega": 0.25, "n": 4}, {"name": "u", "omega": 0.125, "n": 4}],
            "terms": [{"d": 0, "dp": 0, "coef": 1.5, "pow": [0, 0]}, {"d": 1, "dp": 1, "coef": 1.0, "pow": [0, 0]},
                      {"d": 0, "dp": 1, "coef": 0.1, "pow": [0, 1]}],
            "channels": [{"d": 0, "mu": 0, "a": 0.1, "b": 0.5, "l": 0}]}


@pytest.mark.parametrize("method,precision,span", [("cocg", "mixed", 0), ("cocg", "fp64", 0), ("gmres", "fp64", 0),
                                                   ("gmres", "mixed", 0), ("cocg", "fp64", 0x1),
                                                   ("gmres", "mixed", 0x1)])
def test_zero_pivot_is_reported(vbk, method, precision, span):
    model = vbk.Model(_zero_pivot_model())
    opts = vbk.vbk_default_opts(method=method, precision=precision, precond_span=span, tol=1e-10, max_iter=200,
                                max_refine=5)
    with pytest.raises(vbk.VbkError) as err:
        vbk.vbk_solve(model, [1.125], [[0, 0]], opts)
    assert err.value.code == vbk.VBK_ERR_NOT_CONVERGED
    _, st = vbk.vbk_solve(model, [1.125], [[0, 0]], opts, check=False)
    assert [s["status"] for s in st] == ["pivot"]
    # away from the zero pivot the same model converges
    _, st = vbk.vbk_solve(model, [1.16], [[0, 0]], opts)
    assert [s["status"] for s in st] == ["converged"]


def test_non_finite_energies_are_rejected(vbk):
    model = vbk.Model(w.ci2d_model(4))
    for bad in (float("nan"), float("inf")):
        with pytest.raises(vbk.VbkError) as err:
            vbk.vbk_solve(model, [1.0, bad], [[0, 0]])
        assert err.value.code == 1
        x = torch.zeros((1, 1, model.N), dtype=torch.complex128, device="cuda")
        with pytest.raises(vbk.VbkError) as err:
            vbk.vbk_matvec(model, [bad], x)
        assert err.value.code == 1


@pytest.mark.parametrize("resident", [1, 2, 3, 0])
def test_inner_solves_capped_and_restarted_still_converge(vbk, resident):
    """Mixed COCG whose FP32 inner solves stop after a quarter of the iterations an uncapped
    inner solve takes: each FP64 residual restarts the inner solve (the cure for FP32
    stagnation), the refinement takes more steps and still reaches the tolerance."""
    desc = w.ci2d_model(16)
    model = vbk.Model(desc)
    eps = np.array([0.8, 2.9])
    base = dict(method="cocg", precision="mixed", precond_span=0, tol=1e-9, max_refine=400, resident=resident)
    _, st0 = vbk.vbk_solve(model, eps, [[0, 0]], vbk.vbk_default_opts(inner_max_iter=0, **base))
    cap = max(4, max(s["iterations"] for s in st0) // 4)
    psi, st = vbk.vbk_solve(model, eps, [[0, 0]], vbk.vbk_default_opts(inner_max_iter=cap, **base))
    assert all(s["status"] == "converged" for s in st)
    assert max(s["refinements"] for s in st) > max(s["refinements"] for s in st0)
    assert all(s["iterations"] <= cap * (s["refinements"] + 1) for s in st)
    psi = psi.cpu().numpy()
    for e, ei in enumerate(eps):
        E = o.total_energy(desc, ei, [0, 0])
        for mu in range(2):
            rhs = o.phi(desc, E, [0, 0], mu)
            assert o.relative_residual(desc, E, psi[e, 0, mu], rhs) <= 1e-9 * 1.05


def test_uneven_batch_with_several_initial_states(vbk):
    desc = w.ci2d_model(16)
    model = vbk.Model(desc)
    eps = w.eps_grid(4.0, 9)
    vi = w.lowest_levels(desc, 4)
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=0x5, tol=1e-9, max_refine=200)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    its = [s["iterations"] for s in stats]
    assert min(its) < max(its)  # systems retire at different iterations
    psi = psi.cpu().numpy()
    for e in (0, 4, 8):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, eps[e], v)
            for mu in range(2):
                res = o.relative_residual(desc, E, psi[e, i, mu], o.phi(desc, E, v, mu))
                assert res <= 1e-9 * 1.05


@pytest.mark.parametrize("span,resident", [(0, 1), (0, 2), (0, 3), (0, 0), (0x5, 1)])
def test_full_size_batched_sampled(vbk, span, resident):
    """The 80 x 80 basis (N = 12,800) over 256 energies in (0, 3] eV, in the launch configurations
    of the benchmark (Jacobi: one thread block per system, or grid-wide kernels; M^g): every
    system's true residual is checked by the oracle in complex128, and cross sections of sampled
    energies are compared with sparse-LU solutions."""
    spec = w.WORKLOADS["ci2d_batched"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    model = vbk.Model(desc)
    opts = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=span, tol=1e-8, resident=resident)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    assert all(s["status"] == "converged" for s in stats)
    psi_h = psi.cpu().numpy()
    for e in range(0, eps.size, 5):
        E = o.total_energy(desc, eps[e], vi[0])
        A = o.a_matrix(desc, E)
        for mu in range(2):
            rhs = o.phi(desc, E, vi[0], mu)
            res = np.linalg.norm(rhs - A @ psi_h[e, 0, mu]) / np.linalg.norm(rhs)
            assert res <= 1e-8 * 1.05, (e, mu, res)
    sample = [0, 63, 127, 200, 255]
    vf = [[0, 0], [1, 0], [0, 2], [3, 1]]
    sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf).cpu().numpy()
    ref, _ = o.cross_sections(desc, eps[sample], vi, vf)
    np.testing.assert_allclose(sig[sample], ref, rtol=5e-6)
