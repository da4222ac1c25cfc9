"""Host logic of the autotuner (no GPU): class keys and the cache file."""
import pytest

from paper_1304_4327_gb300 import autotune


def test_width_bucket():
    assert [autotune.width_bucket(d) for d in (1, 4, 5, 8, 9, 16, 17, 32, 33, 64)] == \
        [4, 4, 8, 8, 16, 16, 32, 32, 64, 64]
    with pytest.raises(ValueError):
        autotune.width_bucket(65)


def test_problem_class_groups_by_powers_of_two():
    a = autotune.problem_class(1000, 1000, 3, 10, "fp32")
    assert a == autotune.problem_class(1023, 1001, 4, 10, "fp32")
    assert a != autotune.problem_class(1024, 1000, 3, 10, "fp32")
    assert a != autotune.problem_class(1000, 1000, 3, 1, "fp32")
    assert a != autotune.problem_class(1000, 1000, 5, 10, "fp32")
    assert a != autotune.problem_class(1000, 1000, 3, 10, "bf16")


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    key = autotune.problem_class(1000, 1000, 3, 10, "fp32")
    assert key == "d4/r9/q9/k10/fp32"
    t = autotune.Autotuner(path)
    t.table[key] = (16, 64)
    t.save()
    u = autotune.Autotuner(path)
    assert u.table == {key: (16, 64)}
    # a cached class is answered without measuring (no GPU is touched)
    class Pts:
        shape = (1000, 3)
    assert u.choose(Pts(), None, 10, "fp32") == (16, 64)
