"""The FP64 oracle against stored exact solutions (tests/golden/tiny_exact.json):
the minimiser of Eq. 5 and its Eq. 17 adjoint for small seeded problems and a
hand-worked two-DoF case, computed in exact rational arithmetic by
tests/golden/make_golden.py, which uses no solver code."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_exact.json")


def load_cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _rel(x, y):
    x = np.asarray(x, np.float64).ravel()
    y = np.asarray(y, np.float64).ravel()
    if y.size == 0:
        return 0.0
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def test_fixture_is_what_its_script_writes():
    # the stored values come from the committed exact-arithmetic script alone
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(GOLDEN), "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(GOLDEN) as fh:
        stored = json.load(fh)
    assert json.loads(json.dumps(mod.build_document())) == stored


def test_fixture_covers_the_cases_it_claims():
    cases = load_cases()
    names = [c["name"] for c in cases]
    assert "two-dof" in names and len(cases) >= 15
    assert {c["nv"] for c in cases} >= {2, 3, 4, 5}
    assert any(c["m"] == 0 for c in cases) and any(sum(c["active"]) == 0 and c["m"] > 0
                                                     for c in cases)
    two = cases[names.index("two-dof")]
    assert two["a"] == pytest.approx([-5 / 11, 12 / 11], rel=0, abs=1e-15)
    assert two["dJ"][0] == pytest.approx([63 / 121, -72 / 121], rel=0, abs=1e-15)


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_oracle_matches_exact_solution(case):
    M = np.asarray(case["M"], np.float64)
    J = np.asarray(case["J"], np.float64).reshape(case["m"], case["nv"])
    a, act, st, _ = oracle.solve_one(M, J, case["qfrc"], case["aref"], case["D"])
    assert st == 0
    assert np.asarray(act, int).tolist() == case["active"]
    assert _rel(a, case["a"]) <= 1e-10
    dq, dr, dJ, _, _ = oracle.adjoint_one(M, J, case["qfrc"], case["aref"], case["D"], a,
                                          case["g"])
    assert _rel(dq, case["dqfrc"]) <= 1e-10
    assert _rel(dr, case["daref"]) <= 1e-10
    assert _rel(dJ, np.asarray(case["dJ"]).reshape(case["m"], case["nv"])) <= 1e-10
