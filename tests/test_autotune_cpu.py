"""Host logic of the autotuner (no GPU)."""
from paper_1908_05232_b300 import autotune


def test_cache_key_buckets_crowds_by_power_of_two():
    assert autotune.cache_key("B300", 512, 512, 10_000) == "B300|512x512|peds<=16384"
    assert autotune.cache_key("B300", 512, 512, 16_384) == "B300|512x512|peds<=16384"
    assert autotune.cache_key("B300", 512, 512, 16_385) == "B300|512x512|peds<=32768"
    assert autotune.cache_key("B300", 64, 32, 0) == "B300|64x32|peds<=0"


def test_batch_size_classes_split_by_cell_count():
    cells = [1024 * 1024, 128 * 128, 512 * 512, 256 * 256, 768 * 768]
    assert autotune.size_classes(cells, 2) == [1, 0, 0, 0, 1]  # ranks 0-2 small, 3-4 large
    assert autotune.size_classes(cells, 1) == [0] * 5
    assert autotune.size_classes(cells, 5) == [4, 0, 2, 1, 3]
    # ties keep the input order; every class of equal-size members is used
    assert autotune.size_classes([100] * 4, 2) == [0, 0, 1, 1]
    assert autotune.size_classes([], 2) == []


def test_tune_batch_of_nothing_needs_no_gpu():
    assert autotune.tune_batch([]) == {"shapes": [], "us_per_step": 0.0, "uniform": {}, "classes": []}
