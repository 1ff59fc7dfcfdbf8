"""The C ABI library: it builds, loads, exports every entry point include/mka.h declares,
and rejects bad arguments before touching the GPU. No compute call runs here."""
import os
import re

import numpy as np
import pytest

from paper_1202_0098_gb300 import build, mka
from synth import SK_CARBON_LIKE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mka.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mka.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mka_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(mka.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert mka.mka_status_string(mka.MKA_OK) == "ok"
    assert "positive definite" in mka.mka_status_string(mka.MKA_ERR_NOT_SPD)


def test_bad_arguments_are_rejected(lib):
    pos = np.zeros((4, 3))
    with pytest.raises(mka.MkaError) as e:
        mka.mka_build_system(pos, np.array([10.0, 10.0, 10.0]), SK_CARBON_LIKE, "fp64", cluster_radius=6.0)
    assert e.value.status == mka.MKA_ERR_INVALID_ARG          # R >= box / 2
    with pytest.raises(mka.MkaError) as e:
        mka.mka_build_system(pos, np.array([-1.0, 10.0, 10.0]), SK_CARBON_LIKE, "fp64", cluster_radius=2.0)
    assert e.value.status == mka.MKA_ERR_INVALID_ARG
    with pytest.raises(mka.MkaError) as e:
        mka.mka_solve_columns(None, None, mka.solve_params(15, 15))
    assert e.value.status == mka.MKA_ERR_INVALID_ARG


def test_no_gpu_means_cuda_error_not_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    pos = np.random.default_rng(0).random((8, 3)) * 10.0
    with pytest.raises(mka.MkaError) as e:
        mka.mka_build_system(pos, np.array([10.0, 10.0, 10.0]), SK_CARBON_LIKE, "fp64", cluster_radius=3.0)
    assert e.value.status == mka.MKA_ERR_CUDA


def _bsr_case(kind):
    """A 3-atom BSR pattern (every row: its diagonal and its neighbours, ascending), broken one way."""
    row_ptr = np.array([0, 2, 5, 7])
    col = np.array([0, 1, 0, 1, 2, 1, 2])
    if kind == "descending":
        col = np.array([0, 1, 1, 0, 2, 1, 2])
    elif kind == "no_diagonal":
        row_ptr, col = np.array([0, 1, 4, 6]), np.array([1, 0, 1, 2, 1, 2])
    elif kind == "out_of_range":
        col = np.array([0, 1, 0, 1, 3, 1, 2])
    elif kind == "row_ptr":
        row_ptr = np.array([0, 2, 5, 6])
    n = len(col)
    eye = np.broadcast_to(np.eye(4), (n, 4, 4)).copy()
    return row_ptr, col, eye, eye


@pytest.mark.parametrize("kind", ["descending", "no_diagonal", "out_of_range", "row_ptr"])
def test_bad_bsr_input_is_rejected_on_the_host(lib, kind):
    """Malformed caller BSR arrays fail validation before any device work (so also without a GPU)."""
    pos = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0], [3.0, 1.0, 1.0]])
    row_ptr, col, H, S = _bsr_case(kind)
    with pytest.raises(mka.MkaError) as e:
        mka.mka_build_system_bsr(pos, np.array([10.0, 10.0, 10.0]), row_ptr, col, H, S, cluster_radius=2.0)
    assert e.value.status == mka.MKA_ERR_INVALID_ARG


def test_cutoff_beyond_half_the_box_is_rejected(lib):
    from dataclasses import replace
    with pytest.raises(mka.MkaError) as e:
        mka.mka_build_system(np.zeros((4, 3)), np.array([5.0, 5.0, 5.0]), replace(SK_CARBON_LIKE, rc=3.0), "fp64",
                             cluster_radius=2.0)
    assert e.value.status == mka.MKA_ERR_INVALID_ARG
