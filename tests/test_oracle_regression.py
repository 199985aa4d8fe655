"""The oracle's outputs on small seeded inputs against the committed digests
(tests/golden/oracle_regression.txt, written by make_oracle_regression.py):
a change to the oracle's arithmetic shows up here and must be deliberate."""

import importlib.util
import os

from conftest import GOLDEN


def test_oracle_outputs_match_committed_digests():
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(GOLDEN, "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    want = {}
    with open(os.path.join(GOLDEN, "oracle_regression.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, d = (x.strip() for x in line.split("|"))
            want[name] = d
    got = dict(mod.rows())
    assert set(got) == set(want)
    for name, d in got.items():
        assert d == want[name], name
