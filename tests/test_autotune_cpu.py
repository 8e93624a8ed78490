"""Host logic of the autotuner (no GPU)."""
from paper_1908_05232_b300 import autotune


def test_cache_key_buckets_crowds_by_power_of_two():
    assert autotune.cache_key("B300", 512, 512, 10_000) == "B300|512x512|peds<=16384"
    assert autotune.cache_key("B300", 512, 512, 16_384) == "B300|512x512|peds<=16384"
    assert autotune.cache_key("B300", 512, 512, 16_385) == "B300|512x512|peds<=32768"
    assert autotune.cache_key("B300", 64, 32, 0) == "B300|64x32|peds<=0"
