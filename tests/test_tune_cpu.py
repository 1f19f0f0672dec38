"""CPU test of the autotuner's selection: the fastest candidate whose E_c equals
the default setting's wins; failed or disagreeing candidates never do."""
from paper_2405_20258_gb300 import tune


def test_select_fastest_agreeing_candidate():
    grid = {"RPA_TC_NB": ["2", "3"], "RPA_TC_GROUP": ["4", "8"]}
    times = {("2", "4"): 9.0, ("2", "8"): 7.0, ("3", "4"): 5.0, ("3", "8"): 6.0}
    seen = []

    def run(setting):
        seen.append(setting)
        if not setting:
            return {"ec": -1.0, "gemm_ms": 10.0}
        key = (setting["RPA_TC_NB"], setting["RPA_TC_GROUP"])
        if key == ("3", "4"):
            return {"ec": -1.0 + 1e-6, "gemm_ms": times[key]}   # fastest, but E_c moved
        if key == ("2", "4"):
            return {"error": "launch failed"}
        return {"ec": -1.0, "gemm_ms": times[key]}

    best, results = tune.select(grid, run)
    assert seen[0] == {} and len(seen) == 5
    assert best["env"] == {"RPA_TC_NB": "3", "RPA_TC_GROUP": "8"} and best["gemm_ms"] == 6.0
    assert sum("error" in r for r in results) == 1
    assert [r["agrees"] for r in results if "agrees" in r] == [True, True, False, True]


def test_select_without_a_working_candidate():
    best, results = tune.select({"RPA_TC_NB": ["2"]}, lambda s: {"error": "no device"})
    assert best is None and len(results) == 2
