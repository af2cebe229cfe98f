"""CPU-side checks of the CUDA library: it loads, exports every function
include/jk.h declares, rejects bad arguments with error codes, and its
runtime-compiled kernels build for sm_103a with NVRTC (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2507_09772_gb300 import build as jbuild
from paper_2507_09772_gb300 import jk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    jbuild.build()
    return jk.load_library()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "jk.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(jk_\w+)\s*\(", txt, flags=re.M)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(jk.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p()
    rc = lib.jk_init(None, 0, None, 0, None, None, 0, ctypes.byref(h))
    assert rc == jk.JK_ERR_ARG
    assert "NULL" in jk.jk_last_error() or "empty" in jk.jk_last_error()
    assert lib.jk_init(None, 0, None, 0, None, None, 0, None) == jk.JK_ERR_ARG
    assert lib.jk_build(None, None, 1, 1, 1, 1e-13, 0, None, None, None, None) == jk.JK_ERR_ARG
    assert lib.jk_destroy(None) == jk.JK_ERR_ARG
    assert lib.jk_set_option(None, b"tau32", 1.0) == jk.JK_ERR_ARG


def test_unsupported_shell_is_rejected_before_any_device_call(lib):
    shells = np.array([[0, 5, 1, 0, 0, 0]], dtype=np.int32)   # l = 5 > JK_LMAX
    with pytest.raises(jk.JKError) as e:
        jk.jk_init(shells, np.zeros((1, 3)), np.ones(1), np.ones(1))
    assert e.value.code == jk.JK_ERR_UNSUPPORTED


def test_bad_shell_fields_are_rejected(lib):
    shells = np.array([[3, 0, 1, 0, 0, 0]], dtype=np.int32)   # atom index out of range
    with pytest.raises(jk.JKError) as e:
        jk.jk_init(shells, np.zeros((1, 3)), np.ones(1), np.ones(1))
    assert e.value.code == jk.JK_ERR_ARG
    shells = np.array([[0, 0, 1, 0, 0, 0]], dtype=np.int32)
    with pytest.raises(jk.JKError) as e:
        jk.jk_init(shells, np.zeros((1, 3)), -np.ones(1), np.ones(1))   # negative exponent
    assert e.value.code == jk.JK_ERR_ARG


@pytest.mark.parametrize("cls", [
    (0, 0, 0, 0, 6, 6, 6, 6, 0), (1, 0, 1, 0, 3, 1, 3, 1, 0), (1, 1, 1, 1, 1, 1, 1, 1, 0),
    (2, 0, 1, 0, 1, 3, 3, 1, 0), (2, 2, 2, 2, 1, 1, 1, 1, 0), (2, 1, 0, 0, 1, 3, 6, 6, 1),
    (1, 1, 0, 0, 3, 3, 6, 1, 1), (2, 2, 1, 1, 1, 1, 1, 1, 1)])
def test_class_kernels_compile_for_sm103a(lib, cls, tmp_path, monkeypatch):
    monkeypatch.setenv("JK_KERNEL_CACHE", str(tmp_path))
    g, ms = jk.jk_compile_class(*cls[:8], n_dm=1, with_j=1, with_k=1, fp32=cls[8])
    g2, _ = jk.jk_compile_class(*cls[:8], n_dm=1, with_j=1, with_k=1, fp32=cls[8], mode=1)
    assert g2 == g
    assert g >= 1
    assert any(p.suffix == ".bin" for p in tmp_path.iterdir())


def test_compile_rejects_out_of_range(lib):
    with pytest.raises(jk.JKError) as e:
        jk.jk_compile_class(5, 0, 0, 0, 1, 1, 1, 1)
    assert e.value.code == jk.JK_ERR_UNSUPPORTED


def test_compile_basis_builds_every_kernel_of_a_basis(lib, tmp_path, monkeypatch):
    monkeypatch.setenv("JK_KERNEL_CACHE", str(tmp_path))
    shells = np.array([[0, 1, 2, 0, 0, 0], [0, 0, 3, 2, 3, 0]], dtype=np.int32)   # p2, s3
    nk, ms = jk.jk_compile_basis(shells)
    # 3 pair classes: 2 Schwarz kernels each (contracted, primitive) + 6 class pairs
    assert nk == 3 * 2 + 6
    assert len(list(tmp_path.iterdir())) == nk


def _ncart(l):
    return (l + 1) * (l + 2) // 2


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 1, 1, 0), (2, 2, 2, 2), (3, 2, 3, 2),
                                 (3, 3, 3, 3), (4, 4, 2, 2)])
@pytest.mark.parametrize("fp32", [0, 1])
def test_fragment_candidates_are_valid_shapes(lib, cls, fp32):
    """Autotuner candidates: distinct shapes, each g dividing its shell's
    Cartesian size, G <= 256 and at most 64 elements per thread (G = 1 and the
    built-in heuristic's shape excepted, which come first)."""
    c = jk.jk_fragment_candidates(*cls, fp32=fp32, max_candidates=8)
    assert 1 <= len(c) <= 8 and len(set(c)) == len(c)
    nf = [_ncart(l) for l in cls]
    ne = int(np.prod(nf))
    for k, g in enumerate(c):
        assert all(n % x == 0 for n, x in zip(nf, g)), g
        G = int(np.prod(g))
        assert G <= 256
        if k > 0 and G > 1:
            assert ne // G <= 64


def test_fragment_candidates_reject_bad_arguments(lib):
    with pytest.raises(jk.JKError):
        jk.jk_fragment_candidates(5, 0, 0, 0)
    with pytest.raises(jk.JKError):
        jk.jk_fragment_candidates(1, 1, 1, 1, max_candidates=0)


def test_group_split_over_ctas_compiles(lib, tmp_path, monkeypatch):
    """(gg|gg) needs more than 256 threads within the fragment budget: its
    quartets are split over several CTAs (threads per quartet above 256);
    the class kernel and the Schwarz kernels of a g basis compile for sm_103a."""
    monkeypatch.setenv("JK_KERNEL_CACHE", str(tmp_path))
    g, _ = jk.jk_compile_class(4, 4, 4, 4, 1, 1, 1, 1)
    assert g > 256
    shells = np.array([[0, 4, 1, 0, 0, 0]], dtype=np.int32)
    nk, _ = jk.jk_compile_basis(shells)
    assert nk == 1 * 2 + 1
