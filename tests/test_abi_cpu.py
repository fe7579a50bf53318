"""CPU-only checks of the C-ABI library: it loads, exports every entry point that
include/dg.h declares, rejects bad arguments without touching a GPU, and its
reference-element tables agree with numpy's Gauss rule and Legendre roots."""
import os
import re

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

import __graft_entry__ as ge
from paper_1812_08075_gb300 import build as libbuild, dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    libbuild.build()
    return dg.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert "dg_apply" in names and "dg_apply_adjoint" in names and "dg_operator_create" in names
    lib = dg.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(dg.EXPORTED) == names


def test_binding_constants_match_the_header_enums():
    # every DG_* enumerator of include/dg.h has the same value in the Python binding
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dg.h")).read(), flags=re.S)
    found = 0
    for body in re.findall(r"enum\s*\{([^}]*)\}", src):
        for name, val in re.findall(r"\b(DG_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            assert getattr(dg, name) == int(val), name
            found += 1
    assert found >= 20 and dg.DG_VARIANT_DF64 == 4


def test_status_strings_and_argument_errors_without_gpu():
    assert dg.status_string(dg.DG_OK) == "DG_OK"
    assert dg.status_string(dg.DG_ERR_UNSUPPORTED) == "DG_ERR_UNSUPPORTED"
    with pytest.raises(dg.DGError) as e:
        dg.dg_mesh_create(0, 2, 2)
    assert e.value.status == dg.DG_ERR_INVALID_ARG
    assert dg.lib().dg_get_last_error() == dg.DG_ERR_INVALID_ARG
    assert dg.lib().dg_get_last_error() == dg.DG_OK
    m = dg.dg_mesh_create(2, 2, 2)
    pen = dg.dg_penalty(dg.DG_PEN_CONFIG, 0, 2.0)
    for deg, mq, co, st in [
        (0, 0, dg.dg_coefficients(0, 0, 63, 1, 0, 0, 1.0, 1.0, -1.0), dg.DG_ERR_INVALID_ARG),
        (6, 0, dg.dg_coefficients(0, 0, 63, 1, 0, 0, 1.0, 1.0, -1.0), dg.DG_ERR_UNSUPPORTED),
        (2, 2, dg.dg_coefficients(0, 0, 63, 1, 0, 0, 1.0, 1.0, -1.0), dg.DG_ERR_INVALID_ARG),
        (2, 0, dg.dg_coefficients(0, 0, 63, 17, 0, 0, 1.0, 1.0, -1.0), dg.DG_ERR_INVALID_ARG),
        (2, 0, dg.dg_coefficients(0, 0, 64, 1, 0, 0, 1.0, 1.0, -1.0), dg.DG_ERR_INVALID_ARG),
        (2, 0, dg.dg_coefficients(5, 0, 63, 1, 0, 0, 1.0, 1.0, -1.0), dg.DG_ERR_INVALID_ARG),
    ]:
        with pytest.raises(dg.DGError) as e:
            dg.dg_operator_create(m, deg, mq, pen, co)
        assert e.value.status == st
    dg.dg_mesh_destroy(m)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_cuda_path_tables_match_numpy(k):
    t = dg.dg_reference_tables(k)
    m = k + 1
    s, w = npleg.leggauss(m)
    np.testing.assert_allclose(t["gauss_nodes"], (s + 1) / 2, atol=1e-15)
    np.testing.assert_allclose(t["gauss_weights"], w / 2, atol=1e-15)
    if k == 1:
        z = np.array([-1.0, 1.0])
    else:
        z = np.concatenate([[-1], np.sort(npleg.Legendre.basis(k).deriv().roots()), [1]])
    np.testing.assert_allclose(t["gll_nodes"], (z + 1) / 2, atol=1e-14)
    # interpolation reproduces polynomials of degree <= k at the Gauss points
    g, q = t["gll_nodes"], t["gauss_nodes"]
    for d in range(k + 1):
        np.testing.assert_allclose(t["interp"] @ g ** d, q ** d, atol=1e-13)
    # collocated derivative is exact on degree <= m-1, and the end rows evaluate at 0 and 1
    for d in range(m):
        np.testing.assert_allclose(t["dcol"] @ q ** d, d * q ** max(d - 1, 0) if d else 0 * q, atol=1e-12)
        np.testing.assert_allclose(t["end_val"] @ q ** d, [0.0 ** d, 1.0], atol=1e-12)
        np.testing.assert_allclose(t["end_der"] @ q ** d, [d * 0.0 ** max(d - 1, 0) if d else 0, d], atol=1e-11)
