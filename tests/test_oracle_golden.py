"""The oracle against its stored outputs on small seeded cases (tests/golden, written by
tests/golden/make_oracle_golden.py from the oracle alone).  A change to the oracle's
arithmetic fails here and must name the passage of the paper that justifies it; the
stored values are then rewritten by that script.  Integer results (segment counts, hit
primitives) must match exactly; FP64 values to 1e-12 relative (libm and OpenMP reduction
order may differ in the last bits between machines)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

from make_oracle_golden import cases  # noqa: E402


def _close(a, b, rtol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return a.shape == b.shape and np.all(np.abs(a - b) <= rtol * np.max(np.abs(b)) + 1e-300)


def test_oracle_matches_its_stored_outputs():
    with open(os.path.join(HERE, "golden", "oracle_small_cases.json")) as f:
        ref = json.load(f)
    now = cases()
    assert _close(now["fan_latlong"]["dirs"], ref["fan_latlong"]["dirs"], 1e-14)
    assert _close(now["fan_latlong"]["weights"], ref["fan_latlong"]["weights"], 1e-14)
    assert now["open_plane"]["receivers"] == ref["open_plane"]["receivers"]
    for k in ("re", "im"):
        assert _close(now["open_plane"][k], ref["open_plane"][k], 1e-12), k
        assert _close(now["city_sum"][k], ref["city_sum"][k], 1e-12), k
        assert _close(now["city_lossy"][k], ref["city_lossy"][k], 1e-12), k
    assert now["city_trace"] == ref["city_trace"]
    for k in ("grad_gamma", "grad_b", "grad_weight_sum", "grad_weight_norm"):
        assert _close(now["city_adjoint"][k], ref["city_adjoint"][k], 1e-10), k
