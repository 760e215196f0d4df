"""The C-ABI library builds, loads and exports every function include/vbk.h declares; host-only
entry points behave as documented (no GPU needed).

The host level shift is pinned against the oracle's closed form (which is itself pinned
against quadrature), so the library's own Dawson and erfcx code paths (series near zero,
piecewise polynomials, asymptotic expansions) are checked on both sides of threshold.  The
ctypes structures of the binding are checked field by field against the C header compiled by
the host compiler.
"""

import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vbk.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2307_13483_gb300 as vbk

    return vbk


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vbk_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ["vbk_build_model", "vbk_solve", "vbk_cross_sections", "vbk_solve_adjoint", "vbk_free_model"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vbk_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    # the Python binding marshals exactly these names
    assert sorted(lib.EXPORTED) == declared_functions()


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_host_level_shift_matches_oracle(lib, l):
    from oracle import vibronic as o

    for b in (0.25, 0.4, 0.833, 1.7):
        for eps in np.concatenate([np.linspace(-40, -0.01, 23), [-1e-6, 0.0, 1e-6], np.linspace(0.003, 12, 41)]):
            got = lib.vbk_level_shift(eps, 0.13, b, l)
            ref = complex(o.level_shift(np.array([eps]), 0.13, b, l)[0])
            # the upward recursion P_l = -Gamma(l+1/2) b^-(l+1/2) + eps P_(l-1) cancels for eps < 0:
            # both sides lose about (1 + |eps|)^l of relative accuracy there
            cond = (1.0 + abs(eps)) ** (l + 0.5) if eps < 0 else 1.0
            assert abs(got - ref) <= 2e-13 * cond * max(1.0, abs(ref)), (eps, b, l, got, ref)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_double_float_level_shift_matches_the_fp64_closed_form(lib, l):
    """The double-float code the FP32 refinement path's energy tables run (evaluated on the
    host) against the FP64 closed form and the oracle: every branch (Taylor, interpolants,
    asymptotic series; open and closed channels; threshold), relative to the diagonal scale
    (the level shift enters A beside E - E_nu, an eV-sized term)."""
    from oracle import vibronic as o

    for b in (0.25, 0.4, 0.833, 1.7):
        # b eps = 300 reaches the asymptotic series; with l > 0 the upward recursion cancels there
        # (as in FP64, with double-float's shorter significand), far beyond the energies of interest
        far = [300.0 / b] if l == 0 else []
        for eps in np.concatenate([np.linspace(-40, -0.01, 23), [-1e-6, 0.0, 1e-6], np.linspace(0.003, 40, 61),
                                   [0.02, 0.6 / b, 3.0 / b], far]):
            got = lib.vbk_level_shift_df(eps, 0.13, b, l)
            ref = lib.vbk_level_shift(eps, 0.13, b, l)
            orc = complex(o.level_shift(np.array([eps]), 0.13, b, l)[0])
            cond = (1.0 + abs(eps)) ** (l + 0.5) if eps < 0 else 1.0
            scale = max(1.0, abs(ref), abs(eps))  # F enters A beside E - E_nu, of size |eps|
            assert abs(got - ref) <= 2e-14 * cond * scale, (eps, b, l, got, ref)
            assert abs(got - orc) <= 2e-13 * cond * scale, (eps, b, l, got, orc)
            if 0 < b * eps < 80:  # the width, where exp(-b eps) is representable in float
                # exp(-b eps) inherits the absolute error of its argument, ~1e-14 b eps in double-float
                assert abs(got.imag - ref.imag) <= 1.5e-14 * (1.0 + b * eps) * abs(ref.imag), (eps, b, l)


def test_host_level_shift_rejects_bad_arguments(lib):
    with pytest.raises(lib.VbkError):
        lib.vbk_level_shift(1.0, 0.1, -1.0, 0)
    with pytest.raises(lib.VbkError):
        lib.vbk_level_shift(float("nan"), 0.1, 1.0, 0)


def test_default_options(lib):
    o = lib.vbk_default_opts()
    assert (o.method, o.precision, o.precond_span, o.restart) == (lib.VBK_GMRES, lib.VBK_MIXED, 0, 64)
    assert o.tol == 1e-8 and o.inner_tol == 1e-5 and o.check_every == 8 and o.timing == 0 and o.autotune == 1 and o.resident == 1
    assert o.inner_max_iter == 2000 and o.max_iter == 20000 and o.max_refine == 40
    assert o.matvec_variant == -1
    o2 = lib.vbk_default_opts(method="cocg", precision="fp64", tol=1e-10)
    assert (o2.method, o2.precision, o2.tol) == (lib.VBK_COCG, lib.VBK_FP64, 1e-10)


def test_binding_structs_match_the_header(lib, tmp_path):
    """sizeof and every field offset of the ABI structs, from the header compiled by gcc, equal
    those of the binding's ctypes classes (a field added on one side only would shift them)."""
    import ctypes

    structs = {"vbk_term": lib.vbk_term, "vbk_channel": lib.vbk_channel, "vbk_cterm": lib.vbk_cterm,
               "vbk_model_desc": lib.vbk_model_desc, "vbk_opts": lib.vbk_opts, "vbk_stats": lib.vbk_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[name, field] = int(value)
    for name, cls in structs.items():
        assert got[name, "sizeof"] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[name, fname] == getattr(cls, fname).offset, (name, fname)


def test_binding_constants_match_header(lib):
    """Every #define of the header that the binding also names has the same value."""
    text = open(HEADER).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(VBK_[A-Z_0-9]+)\s+(-?\d+)", text)}
    shared = [k for k in defs if hasattr(lib, k)]
    assert "VBK_MATVEC_NVARIANTS" in shared and "VBK_OK" in shared
    for k in shared:
        assert getattr(lib, k) == defs[k], k


def test_status_strings(lib):
    assert lib.vbk_status_str(0) == "ok"
    assert lib.vbk_status_str(4) == "not converged"
    assert lib.vbk_sys_status_str(2) == "breakdown"
    assert lib.vbk_status_str(99) == "unknown status"


def test_build_without_device_reports_no_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import workloads

    with pytest.raises(lib.VbkError) as ei:
        lib.Model(workloads.ci2d_model(4))
    assert ei.value.code == 6


def test_autograd_parameter_ids_match_the_oracle(lib):
    """The autograd wrapper maps parameter ids to model values exactly as the oracle does: U terms,
    a / b of channels, then coupling-polynomial coefficients channel by channel (Table II model)."""
    import workloads
    from oracle import vibronic as o
    from paper_2307_13483_gb300.autograd import _with_values

    desc = workloads.gen_ecd_model(3, 3)
    n = len(desc["terms"]) + 2 * len(desc["channels"]) + sum(len(c["terms"]) for c in desc["channels"])
    for tid in range(n):
        value = 0.5 + 0.01 * tid
        assert _with_values(desc, [tid], [value]) == o.with_parameter(desc, tid, value), tid


def test_malformed_models_are_rejected_before_any_device_work(lib):
    """vbk_build_model checks the description before it touches a device: each malformed model
    returns VBK_ERR_INVALID_ARG (1) on any machine, with or without a GPU."""
    import copy
    import ctypes

    import workloads

    base = workloads.ci2d_model(4)
    cases = {}
    m = copy.deepcopy(base)
    m["n_states"] = 0
    cases["no states"] = m
    m = copy.deepcopy(base)
    m["modes"][1]["omega"] = 0.0
    cases["omega 0"] = m
    m = copy.deepcopy(base)
    m["modes"][0]["n"] = 0
    cases["empty basis"] = m
    m = copy.deepcopy(base)
    m["terms"][0]["pow"] = [9, 0]
    cases["power 9"] = m
    m = copy.deepcopy(base)
    m["terms"].append({"d": 1, "dp": 0, "coef": 0.1, "pow": [0, 1]})
    cases["d > dp"] = m
    m = copy.deepcopy(base)
    m["terms"][0]["coef"] = float("nan")
    cases["nan coefficient"] = m
    m = copy.deepcopy(base)
    m["channels"][0]["b"] = 0.0
    cases["b 0"] = m
    m = copy.deepcopy(base)
    m["channels"].append(copy.deepcopy(m["channels"][0]))
    cases["state twice on one wave"] = m
    m = workloads.gen_ecd_model(3, 3)
    m["channels"][1]["l"] = 1
    cases["q-dependent wave with two l"] = m
    m = workloads.co2_polar_model(basis=(2, 3, 3, 2))
    m["terms"].append({"d": 0, "dp": 0, "coef": 0.1, "pow": [0, 1, 0, 0], "raise": [0, 1, 0, 0], "lower": [0, 0, 0, 0]})
    cases["power of q and ladder monomial on one mode"] = m
    m = workloads.co2_polar_model(basis=(2, 3, 3, 2))
    m["terms"].append({"d": 0, "dp": 1, "coef": 0.1, "pow": [0, 0, 0, 0], "raise": [0, 9, 0, 0], "lower": [0, 0, 0, 0]})
    cases["ladder power 9"] = m
    m = workloads.gen_ecd_model(3, 3)
    m["channels"][0]["terms"][1]["pow"] = [0, 0, 1]
    cases["coupling power beyond n_modes"] = m
    for name, desc in cases.items():
        with pytest.raises(lib.VbkError) as ei:
            lib.Model(desc)
        assert ei.value.code == 1, name
    # a coupling term that names no channel (built directly: the dictionaries cannot express it)
    d = lib.vbk_model_desc()
    d.n_states, d.n_modes = 1, 1
    d.n_basis[0], d.omega[0] = 4, 0.2
    ch = (lib.vbk_channel * 1)()
    ch[0].d, ch[0].mu, ch[0].a, ch[0].b, ch[0].l = 0, 0, 0.1, 1.0, 0
    ct = (lib.vbk_cterm * 1)()
    ct[0].channel, ct[0].coef = 3, 1.0
    d.n_terms, d.n_channels, d.channels, d.n_cterms, d.cterms = 0, 1, ch, 1, ct
    h = ctypes.c_void_p()
    assert lib._lib.vbk_build_model(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "no channel" in lib.vbk_last_error()


def test_every_workload_model_passes_validation(lib):
    """Without a GPU the build stops at the device check, after the description checks: every
    model the workloads define (q-independent and q-dependent couplings, 1 to 4 modes, up to
    4 states) gets that far, i.e. reports VBK_ERR_NO_DEVICE rather than an invalid argument."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import workloads

    models = [workloads.ci2d_model(5), workloads.ci2d_model(5, extra_terms=True), workloads.ecd86_model(4, 6),
              workloads.gen_ecd_model(5, 4), workloads.co2_like_model(basis=(3, 3, 3, 2))]
    one_mode = {"n_states": 1, "modes": [{"name": "x", "omega": 0.2, "n": 7}], "terms": [],
                "channels": [{"d": 0, "mu": 0, "a": 0.1, "b": 1.0, "l": 0,
                              "terms": [{"coef": 1.0, "pow": [0]}, {"coef": 0.3, "pow": [2]}]}]}
    four_states = workloads.ci2d_model(3)
    four_states["n_states"] = 4
    four_states["channels"] += [{"d": 2, "mu": 0, "a": 0.1, "b": 1.0, "l": 0}, {"d": 3, "mu": 1, "a": 0.1, "b": 1.0, "l": 0}]
    for desc in models + [one_mode, four_states]:
        with pytest.raises(lib.VbkError) as ei:
            lib.Model(desc)
        assert ei.value.code == 6, (desc.get("name"), lib.vbk_last_error())
