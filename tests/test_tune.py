"""Lane-count autotuner, host logic (CPU): candidate filtering, the choice by
median with ties to fewer lanes, rank classes and table keys, and the JSON
table's round trip.  The timing itself is a function passed in; here a fake
one with known costs."""
import json

import pytest

from paper_2607_06021_gb300 import tune


def test_rank_class_and_key():
    assert [tune.rank_class(r) for r in (0, 1, 2, 3, 20, 32, 33)] == [1, 1, 2, 4, 32, 32, 64]
    assert tune.table_key("mixed", 4095, 20, 1024) == "mixed/n4095/rf32/b1024"
    assert tune.table_key("mixed", 4095, 17, 1024) == tune.table_key("mixed", 4095, 32, 1024)


def test_candidates_leave_no_lane_empty():
    assert tune.candidate_lanes(1024) == [1, 2, 4, 8]
    assert tune.candidate_lanes(3) == [1, 2]
    assert tune.candidate_lanes(6, (8, 4, 4, 0, -1, 2)) == [2, 4]


def test_choice_by_median_with_ties_to_fewer_lanes():
    # median, not mean: one slow outlier does not decide
    assert tune.choose({1: [10.0, 10.0, 10.0], 4: [8.0, 8.0, 100.0]}) == 4
    # within 1% of the fastest: the fewest lanes win
    assert tune.choose({2: [100.5], 4: [100.0], 8: [99.8]}) == 2
    assert tune.choose({2: [103.0], 4: [100.0], 8: [99.8]}) == 4
    with pytest.raises(ValueError):
        tune.choose({4: []})


def test_tune_lanes_times_every_candidate_once():
    cost = {1: 300.0, 2: 220.0, 4: 200.0, 8: 230.0}
    seen = []

    def measure(lanes):
        seen.append(lanes)
        return [cost[lanes], cost[lanes] * 1.001, cost[lanes] * 0.999]

    lanes, times = tune.tune_lanes(measure, 1024)
    assert lanes == 4 and sorted(seen) == [1, 2, 4, 8]
    assert set(times) == {1, 2, 4, 8} and len(times[4]) == 3


def test_table_round_trip(tmp_path):
    path = str(tmp_path / "lanes.json")
    t = tune.TuneTable(path)
    assert t.get("mixed", 4095, 20, 1024) is None
    t.put("mixed", 4095, 20, 1024, 4, {1: [300.0], 4: [200.0, 210.0, 190.0]})
    t.save()
    data = json.load(open(path))
    assert data["mixed/n4095/rf32/b1024"] == {"lanes": 4, "ms": {"1": 300.0, "4": 200.0}}
    t2 = tune.TuneTable(path)
    assert t2.get("mixed", 4095, 24, 1024) == 4  # same rank class
    assert t2.get("fp64", 4095, 20, 1024) is None
    t2.put("mixed", 4095, 20, 1024, 2, {2: [150.0]})
    assert t2.get("mixed", 4095, 20, 1024) == 2


def test_configs_with_loop_placement():
    # (lanes, device loop): every candidate timed once; ties go to the smallest
    # configuration (fewest lanes, then host loops)
    cost = {(1, False): 300.0, (2, False): 220.0, (4, False): 200.0, (8, False): 230.0,
            (1, True): 260.0, (2, True): 199.5, (4, True): 210.0}
    seen = []

    def measure(cfg):
        seen.append(cfg)
        return [cost[cfg]]

    cfg, times = tune.tune_configs(measure, 1024)
    assert cfg == (2, True) and sorted(seen) == sorted(cost)
    assert tune.choose({(4, False): [100.0], (4, True): [100.5]}) == (4, False)
    assert tune.candidate_configs(3) == [(1, False), (1, True), (2, False), (2, True)]
    assert tune.config_name((4, True)) == "4d" and tune.config_name(2) == "2"


def test_table_round_trip_with_loop_placement(tmp_path):
    path = str(tmp_path / "cfg.json")
    t = tune.TuneTable(path)
    t.put("mixed", 4095, 20, 256, (2, True), {(2, True): [150.0], (4, False): [160.0]}, {"gpu": "x"})
    t.save()
    data = json.load(open(path))
    assert data["mixed/n4095/rf32/b256"] == {"lanes": 2, "loop_on_device": True, "ms": {"2d": 150.0, "4": 160.0},
                                             "gpu": "x"}
    t2 = tune.TuneTable(path)
    assert t2.get_config("mixed", 4095, 20, 256) == (2, True) and t2.get("mixed", 4095, 20, 256) == 2


def test_shape_descent_times_each_value_with_the_best_so_far():
    # gemm rows per thread: 1 is faster; DST threads: 512 is faster only with rpt 1
    def cost(sh):
        c = 100.0 if sh["gemm_rows_per_thread"] == 2 else 80.0
        if sh["dst_cta_threads"] == 512 and sh["gemm_rows_per_thread"] == 1:
            c -= 5.0
        if sh["dst_cta_threads"] == 1024:
            c += 3.0
        return c

    seen = []

    def measure(sh):
        seen.append(dict(sh))
        return [cost(sh)] * 3

    best, times = tune.tune_shapes(measure)
    assert best == {"gemm_rows_per_thread": 1, "dst_cta_threads": 512}
    # first knob timed at the other's first value, second at the first's best
    assert seen[:2] == [{"gemm_rows_per_thread": 2, "dst_cta_threads": 256},
                        {"gemm_rows_per_thread": 1, "dst_cta_threads": 256}]
    assert all(s["gemm_rows_per_thread"] == 1 for s in seen[2:]) and len(seen) == 5
    assert set(times) == {"gemm_rows_per_thread", "dst_cta_threads"}


def test_shape_ties_go_to_the_first_listed_value():
    best, _ = tune.tune_shapes(lambda sh: [100.0 + 0.5 * (sh["dst_cta_threads"] == 256)])
    assert best == {"gemm_rows_per_thread": 2, "dst_cta_threads": 256}  # within 1%: first listed
    assert tune.choose_first({1: [100.0], 2: [99.5]}, (2, 1)) == 2
    assert tune.choose_first({1: [90.0], 2: [99.5]}, (2, 1)) == 1


def test_table_keeps_the_shapes(tmp_path):
    path = str(tmp_path / "t.json")
    t = tune.TuneTable(path)
    assert t.get_shapes("mixed", 4095, 20, 1024) == {"gemm_rows_per_thread": 0, "dst_cta_threads": 0}
    t.put("mixed", 4095, 20, 1024, (8, False), {(8, False): [1.0]},
          {"gemm_rows_per_thread": 1, "dst_cta_threads": 512})
    t.save()
    t2 = tune.TuneTable(path)
    assert t2.get_shapes("mixed", 4095, 20, 1024) == {"gemm_rows_per_thread": 1, "dst_cta_threads": 512}
    assert t2.get_config("mixed", 4095, 20, 1024) == (8, False)


def test_lowrank_difference_of_results():
    torch = pytest.importorskip("torch")
    g = torch.Generator().manual_seed(3)
    U = torch.linalg.qr(torch.randn(200, 6, generator=g, dtype=torch.float64))[0]
    V = torch.linalg.qr(torch.randn(200, 6, generator=g, dtype=torch.float64))[0]
    S = torch.tensor([6.0, 5.0, 4.0, 3.0, 2.0, 1.0], dtype=torch.float64)
    assert tune.lowrank_rel_diff((U, S, V), (U.clone(), S.clone(), V.clone())) == 0.0
    # sign flips of a singular pair leave the product unchanged
    Uf, Vf = U.clone(), V.clone()
    Uf[:, 2] *= -1
    Vf[:, 2] *= -1
    assert tune.lowrank_rel_diff((U, S, V), (Uf, S, Vf)) < 1e-7
    # a 0.1% change of every singular value is a 0.1% change of the product
    d = tune.lowrank_rel_diff((U, S, V), (U, S * 1.001, V))
    assert abs(d - 1e-3) < 1e-6
    # a dropped last pair: ||1|| / ||(6..1)||
    d = tune.lowrank_rel_diff((U, S, V), (U[:, :5], S[:5], V[:, :5]))
    assert abs(d - 1.0 / float(torch.sqrt((S * S).sum()))) < 1e-7
