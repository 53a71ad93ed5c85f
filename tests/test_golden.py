"""Fixtures that restate values the paper fixes (status vocabulary, quality gates)."""
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_status_vocabulary_has_the_six_paper_statuses_plus_deadline():
    rows = _rows("status_vocabulary.txt")
    codes = [int(r[0]) for r in rows]
    assert codes == list(range(7))
    names = [r[1] for r in rows]
    assert names[0] == "CERTIFIED" and names[2] == "TIMEOUT" and names[4] == "NO_FEASIBLE_RETURN"


def test_quality_gates_are_the_papers():
    gates = {r[0]: float(r[1]) for r in _rows("quality_gates.txt")}
    assert gates["paper_budget"] == 1e-4
    assert gates["paper_bound"] == 1e-6
    assert gates["kkt_all"] <= gates["paper_bound"]
