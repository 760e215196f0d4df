"""Block preconditioners whose chains have a half bandwidth p > 16 (Sec. III.B: the CO2 model's
blocks span the states and the two-dimensional bend, 3 * 20 * 20 = 1200 unknowns with p = 120).

They are factored by one thread block per preconditioner block and solved by one warp per
(system, block); the tests compare z = B^-1 r with the oracle's sparse direct solve of the
block-diagonal section of A, run every Krylov method through them, and solve the full-size
CO2-like model (N = 432,000) at 3 eV, where the oracle checks the true residual in complex128.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as w  # noqa: E402
from oracle import vibronic as o  # noqa: E402

pytestmark = pytest.mark.gpu

SPAN_STATES_BEND = 0x1 | 0x4 | 0x8  # d, bend x, bend y of the CO2-like model


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


def ci2d_long_chain(n_g, n_u, extra):
    desc = w.ci2d_model(8, extra_terms=extra)
    desc["modes"][0]["n"], desc["modes"][1]["n"] = n_g, n_u
    return desc


# (model, span): chain half bandwidths 24 (CO2-like 5x4x4x3, chain d + 3 n_by + 12 n_bx),
# 60 (CI2D with q_g^3 terms, chain d + 2 n_u + 20 n_g) and 160 (the widest supported band:
# q_g^2 over a chain d + 2 n_u + 80 n_g)
WIDE_CASES = {
    "co2_small": (lambda: w.co2_like_model(basis=(5, 4, 4, 3)), SPAN_STATES_BEND),
    "ci2d_cubic": (lambda: ci2d_long_chain(9, 10, True), 0x7),
    "ci2d_p160": (lambda: ci2d_long_chain(5, 40, False), 0x7),
}


@pytest.mark.parametrize("case", list(WIDE_CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wide_band_precond_parity(vbk, case, precision):
    make, span = WIDE_CASES[case]
    desc = make()
    model = vbk.Model(desc)
    rng = np.random.default_rng(5)
    E = np.array([1.7, 3.2, 4.4])
    nvec = 3  # 9 systems: the last group of warps is ragged
    r = rand_vectors(rng, (E.size, nvec, model.N))
    z = vbk.vbk_precond_apply(model, E, torch.tensor(r, device="cuda"), span,
                              precision=0 if precision == "fp64" else 1).cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 5e-5
    for e in range(E.size):
        for k in range(nvec):
            ref = o.precond_apply(desc, E[e], span, r[e, k])
            assert np.linalg.norm(z[e, k] - ref) <= tol * np.linalg.norm(ref), (case, e, k)


def test_band_wider_than_supported_is_rejected(vbk):
    desc = ci2d_long_chain(5, 41, False)  # q_g^2 across a chain d + 2 n_u + 82 n_g: p = 164
    model = vbk.Model(desc)
    r = torch.zeros((1, 1, model.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(vbk.VbkError) as ei:
        vbk.vbk_precond_apply(model, [2.0], r, 0x7)
    assert ei.value.code == 5


@pytest.mark.parametrize("method,precision", [("cocg", "mixed"), ("cocg", "fp64"), ("gmres", "mixed"), ("gmres", "fp64")])
def test_wide_band_solve_parity(vbk, method, precision):
    desc = w.co2_like_model(basis=(6, 5, 5, 4))
    model = vbk.Model(desc)
    eps = np.array([0.8, 3.0])
    vi = [[0, 0, 0, 0], [1, 0, 0, 0]]
    opts = vbk.vbk_default_opts(method=method, precision=precision, precond_span=SPAN_STATES_BEND, tol=1e-10,
                                restart=48, max_iter=20000, max_refine=200)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    psi = psi.cpu().numpy()
    nmu = model.n_mu
    for e, ei in enumerate(eps):
        for i, v in enumerate(vi):
            E = o.total_energy(desc, ei, v)
            for mu in range(nmu):
                st = stats[(e * len(vi) + i) * nmu + mu]
                assert st["status"] == "converged", st
                res = o.relative_residual(desc, E, psi[e, i, mu], o.phi(desc, E, v, mu))
                assert res <= 1e-10 * 1.05, (e, i, mu, res)


def test_co2_like_full_size(vbk):
    """3 states x 30 x 20 x 20 x 12 oscillator functions (N = 432,000) at eps_i = 3 eV, v_i = 0,
    all three partial waves, COCG with the states x bend blocks.  This synthetic model needs
    about 2,700 COCG iterations; complex-FP32 COCG stagnates on it, so the solve runs in FP64."""
    spec = w.WORKLOADS["co2_like"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    model = vbk.Model(desc)
    assert model.N == 432000
    opts = vbk.vbk_default_opts(method="cocg", precision="fp64", precond_span=SPAN_STATES_BEND, tol=1e-8,
                                max_iter=20000, max_refine=100)
    psi, stats = vbk.vbk_solve(model, eps, vi, opts)
    assert all(s["status"] == "converged" for s in stats), stats
    psi = psi.cpu().numpy()
    E = o.total_energy(desc, eps[0], vi[0])
    A = o.a_matrix(desc, E)
    for mu in range(model.n_mu):
        rhs = o.phi(desc, E, vi[0], mu)
        res = np.linalg.norm(rhs - A @ psi[0, 0, mu]) / np.linalg.norm(rhs)
        assert res <= 1e-8 * 1.05, (mu, res)
    # the preconditioner at full size: B z = r for the oracle's block-diagonal section B
    rng = np.random.default_rng(9)
    r = rand_vectors(rng, (1, 2, model.N))
    z = vbk.vbk_precond_apply(model, [E], torch.tensor(r, device="cuda"), SPAN_STATES_BEND).cpu().numpy()
    B = o.block_diagonal(desc, E, SPAN_STATES_BEND)
    for k in range(2):
        assert np.linalg.norm(B @ z[0, k] - r[0, k]) <= 1e-10 * np.linalg.norm(r[0, k])
