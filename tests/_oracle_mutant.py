"""pytest plugin for the mutation tests: points the ``oracle`` package at a
mutated copy of ``sta_oracle.c`` (path in ORACLE_MUTANT_SRC), compiled on
first use into a library beside that copy.  Loaded with ``-p`` by
test_oracle_mutants.py only; without the variable it changes nothing."""
import os

import oracle

_src = os.environ.get("ORACLE_MUTANT_SRC")
if _src:
    oracle._SRC = _src
    oracle._LIB = os.path.join(os.path.dirname(_src), "liboracle_mutant.so")
    oracle._lib = None
