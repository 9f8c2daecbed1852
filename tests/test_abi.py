"""The C-ABI library builds for sm_103a (nvcc cross-compiles without a GPU),
loads, and exports every entry point include/bodex.h declares."""
import ctypes
import os
import re

import pytest

from paper_2412_16490_gb300 import _binding, _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bodex.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(bodex_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("bodex_hand_create", "bodex_fk_contacts", "bodex_qp_solve_batch", "bodex_energy_grad",
                 "bodex_step"):
        assert name in syms
    assert set(syms) <= set(_binding.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    lib.bodex_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bodex_version()


def test_invalid_arguments_are_rejected_without_a_gpu():
    L = _binding.load()
    h = ctypes.c_void_p()
    assert L.bodex_hand_create(None, ctypes.byref(h)) == _binding.BODEX_ERR_INVALID
    assert b"null" in L.bodex_last_error()
    p = _binding.bodex_qp_params(0.5, 1.0, 9.0, 0.1, 1e-6, 1.6, 0.0, 0.0, 10, 5, 0, 0)
    # gamma = 9 > m = 4: infeasible, reported before any device work
    rc = L.bodex_qp_solve_batch(None, 0, 4, None, 6, ctypes.byref(p), None, None, None, None, None, None,
                                None, None)
    assert rc == _binding.BODEX_ERR_INFEASIBLE
    p.gamma = 0.5
    rc = L.bodex_qp_solve_batch(None, 0, 7, None, 6, ctypes.byref(p), None, None, None, None, None, None,
                                None, None)
    assert rc in (_binding.BODEX_ERR_INVALID, _binding.BODEX_ERR_INFEASIBLE)
