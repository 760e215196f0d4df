"""vbk_matvec_noalloc: the operator apply for callers that cannot allocate device memory.

Such callers (a process whose device memory another framework has already reserved, a
real-time loop that allows no allocation after start-up) get the FP64 operator from a fixed
scratch array inside the library.  This file runs last so that a failure here never hides
the other tests; it also passes when run alone in a fresh process.
"""

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


def test_noalloc_matches_matvec_on_two_calls_in_a_row(vbk):
    desc = w.ci2d_model(9, extra_terms=True)
    desc["modes"][0]["n"], desc["modes"][1]["n"] = 37, 29
    model = vbk.Model(desc)
    rng = np.random.default_rng(21)
    for E in (np.array([0.35, 2.6, 4.1]), np.array([1.7, 3.3])):
        x = torch.tensor(rng.standard_normal((E.size, 2, model.N)) + 1j * rng.standard_normal((E.size, 2, model.N)),
                         device="cuda")
        ref = vbk.vbk_matvec(model, E, x, precision=vbk.VBK_FP64).cpu().numpy()
        y = torch.full_like(x, complex(float("nan"), 0.0))
        got = vbk.vbk_matvec_noalloc(model, E, x, y).cpu().numpy()
        # the tolerance of the FP64 operator parity tests
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
        assert np.abs(got - ref).max() <= 4e-13 * np.abs(ref).max()


def test_noalloc_matches_the_oracle_operator(vbk):
    """Against the oracle's sparse complex128 A(E) (an independent build of the operator), on a
    ragged basis, at energies with open and closed channels, two calls in a row."""
    desc = w.ci2d_model(9, extra_terms=True)
    desc["modes"][0]["n"], desc["modes"][1]["n"] = 23, 17
    model = vbk.Model(desc)
    rng = np.random.default_rng(5)
    for E in (np.array([0.2, 1.9, 3.7]), np.array([2.8])):
        xh = rng.standard_normal((E.size, 2, model.N)) + 1j * rng.standard_normal((E.size, 2, model.N))
        x = torch.tensor(xh, device="cuda")
        y = torch.full_like(x, complex(float("nan"), 0.0))
        got = vbk.vbk_matvec_noalloc(model, E, x, y).cpu().numpy()
        for e in range(E.size):
            A = o.a_matrix(desc, float(E[e]))
            for v in range(2):
                ref = A @ xh[e, v]
                assert np.linalg.norm(got[e, v] - ref) <= 1e-13 * np.linalg.norm(ref)


def test_noalloc_rejects_q_dependent_couplings(vbk):
    model = vbk.Model(w.gen_ecd_model(6, 5))
    x = torch.zeros((1, 1, model.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(vbk.VbkError) as err:
        vbk.vbk_matvec_noalloc(model, np.array([1.0]), x, torch.empty_like(x))
    assert err.value.code == 5  # VBK_ERR_UNSUPPORTED


def test_noalloc_rejects_more_than_4096_vectors(vbk):
    model = vbk.Model(w.ci2d_model(3))  # N = 18: the bytes fit, the vector count does not
    x = torch.zeros((1, 4097, model.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(vbk.VbkError) as err:
        vbk.vbk_matvec_noalloc(model, np.array([1.0]), x, torch.empty_like(x))
    assert err.value.code == 1 and "4096" in str(err.value)
    x = torch.ones((1, 4096, model.N), dtype=torch.complex128, device="cuda")
    y = vbk.vbk_matvec_noalloc(model, np.array([1.0]), x, torch.empty_like(x))
    ref = vbk.vbk_matvec(model, np.array([1.0]), x, precision=vbk.VBK_FP64)
    assert float((y - ref).abs().max()) <= 1e-13 * float(ref.abs().max())


def test_noalloc_rejects_requests_beyond_its_scratch(vbk):
    model = vbk.Model(w.ci2d_model(80))  # N = 12,800: 16 energies need 3.3 MB, 64 need 13 MB > 8 MiB
    x = torch.zeros((64, 1, model.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(vbk.VbkError) as err:
        vbk.vbk_matvec_noalloc(model, np.linspace(0.1, 3.0, 64), x, torch.empty_like(x))
    assert err.value.code == 1 and "scratch" in str(err.value)
