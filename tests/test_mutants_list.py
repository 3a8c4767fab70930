"""The mutation check's list (tests/mutants.py) still matches the oracle's sources:
every planted mistake's text occurs as often as the list says, every expected outcome is
one of the three kinds, and every expected survivor that is not precision-only has its
reason written down."""
import os

from tests import mutants

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_mutant_pattern_matches_its_source():
    texts = {}
    for name, path, old, new, count, expect in mutants.MUTANTS:
        if path not in texts:
            texts[path] = open(os.path.join(ROOT, path)).read()
        assert texts[path].count(old) == count, name
        assert old != new, name
        assert expect in ("killed", "equivalent", "precision"), name
        if expect == "equivalent":
            assert name in mutants.EQUIVALENT, name
    names = [m[0] for m in mutants.MUTANTS]
    assert len(names) == len(set(names))
    assert set(mutants.EQUIVALENT) <= set(names)
