"""The oracle against its stored results (tests/golden/oracle_regression.json, written by
tests/golden/make_golden.py from oracle/ alone): a change to the oracle's arithmetic
must show up here and be regenerated on purpose, with the passage that justifies it.
Integers (iteration counts, stream lengths, stream checksums, sample indices) must
match exactly; floating-point values to 1e-10 relative (the oracle is compiled without
FMA contraction, so only libm may differ between hosts)."""
import json
import os

import pytest

from golden import make_golden as G

HERE = os.path.dirname(os.path.abspath(__file__))
STORED = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))


def _compare(got, want, path):
    if isinstance(want, dict):
        assert set(got) == set(want), path
        for k in want:
            _compare(got[k], want[k], f"{path}.{k}")
    elif isinstance(want, list):
        assert len(got) == len(want), path
        for i, (a, b) in enumerate(zip(got, want)):
            _compare(a, b, f"{path}[{i}]")
    elif isinstance(want, bool) or isinstance(want, int):
        assert got == want, (path, got, want)
    elif isinstance(want, float):
        assert abs(got - want) <= 1e-10 * abs(want) + 1e-14, (path, got, want)
    else:
        assert got == want, path


@pytest.mark.parametrize("name", sorted(G.CASES))
def test_oracle_reproduces_stored_values(name):
    cite, fn = G.CASES[name]
    want = STORED["cases"][name]
    assert want["cite"] == cite
    _compare(fn(), want["values"], name)
