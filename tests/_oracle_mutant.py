"""pytest plugin for the mutation tests: points the ``oracle`` package at a
mutated copy of ``sta_oracle.c`` (path in ORACLE_MUTANT_SRC), compiled on
first use into a library beside that copy, or replaces the package by a
mutated copy of its Python module (path in ORACLE_MUTANT_PY) that drives the
unmutated C oracle.  Loaded with ``-p`` by test_oracle_mutants.py only;
without the variables it changes nothing."""
import os

import oracle

_src = os.environ.get("ORACLE_MUTANT_SRC")
if _src:
    oracle._SRC = _src
    oracle._LIB = os.path.join(os.path.dirname(_src), "liboracle_mutant.so")
    oracle._lib = None

_py = os.environ.get("ORACLE_MUTANT_PY")
if _py:
    import importlib.util
    import sys

    _spec = importlib.util.spec_from_file_location("oracle", _py)
    _mod = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(_mod)
    _mod._SRC, _mod._LIB, _mod._lib = oracle._SRC, oracle._LIB, None
    sys.modules["oracle"] = _mod
