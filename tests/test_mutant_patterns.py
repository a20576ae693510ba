"""The mutation check (tests/oracle_mutants.py) plants each mistake by exact
text replacement; every text must occur exactly once in the current oracle,
or the check would silently test nothing for that mutant."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _mutants():
    spec = importlib.util.spec_from_file_location("oracle_mutants",
                                                  os.path.join(HERE, "oracle_mutants.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.MUTANTS


@pytest.mark.parametrize("mutant", _mutants(), ids=lambda m: m[0])
def test_mutant_text_occurs_once(mutant):
    name, rel, old, new, _ = mutant
    with open(os.path.join(ROOT, rel)) as f:
        src = f.read()
    assert src.count(old) == 1
    assert old != new


def test_mutant_names_are_unique():
    names = [m[0] for m in _mutants()]
    assert len(names) == len(set(names))
