"""The oracle against its stored reference values (tests/golden/oracle_values.json,
written by tests/golden/make_oracle_golden.py from the oracle alone).  A mismatch
means the oracle's arithmetic changed: regenerate the file only in a commit that
names the passage of the paper justifying the change."""
import json
import os

import numpy as np

from tests.golden.make_oracle_golden import values

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_stored_values():
    with open(os.path.join(HERE, "golden", "oracle_values.json")) as f:
        stored = json.load(f)
    now = values()
    assert sorted(now) == sorted(stored)
    for key, ref in stored.items():
        cur = now[key]
        if key.startswith("tables_"):
            for field in ("tau", "D", "b"):
                assert np.allclose(cur[field], ref[field], rtol=0, atol=1e-14), (key, field)
        else:
            assert cur["status"] == ref["status"] and cur["iterations"] == ref["iterations"], key
            th, th_ref = np.array(cur["theta"]), np.array(ref["theta"])
            assert np.max(np.abs(th - th_ref) / np.abs(th_ref)) < 1e-9, key
            assert abs(cur["phi"] - ref["phi"]) < 1e-9 * abs(ref["phi"]), key
