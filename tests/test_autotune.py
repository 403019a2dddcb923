"""Host logic of the autotuner (CPU): candidate chunk lengths and cache lookup."""
import math

from paper_2602_05017_gb300 import autotune, inputs


def test_candidates_respect_the_kernel_limits():
    for n in range(1, 385):
        c = autotune.candidates(n)
        assert c[-1] == n, n  # whole lines are always a candidate
        for m in c[:-1]:
            assert m < n
            assert math.ceil(n / m) <= autotune.MAX_CHUNKS
            assert m <= autotune.MAX_CHUNK


def test_tile_shapes_use_nearest_class_and_stay_valid():
    cache = {"classes": {"64,4": {"m": [8, 16, 16]}, "192,2": {"m": [24, 24, 24]},
                         "128,1": {"m": [-1, -1, 24]}}}
    envs = [inputs.Workload("a", 70, 70, 70, 4, 20.0, 0.01, [1.0] * 4, [0.0] * 4, 1),
            inputs.Workload("b", 190, 190, 190, 2, 20.0, 0.01, [1.0] * 2, [0.0] * 2, 1),
            inputs.Workload("c", 100, 100, 100, 8, 20.0, 0.01, [1.0] * 8, [0.0] * 8, 1),
            inputs.Workload("d", 120, 130, 125, 1, 20.0, 0.01, [1.0], [0.0], 1)]
    shapes = autotune.tile_shapes(envs, cache)
    assert shapes[0] == [9, 16, 16]   # 70 voxels need >= 9 per chunk
    assert shapes[1] == [24, 24, 24]
    assert shapes[2] == [0, 0, 0]     # no class: library default
    assert shapes[3] == [120, 130, 24]  # whole lines: the environment's own lengths


def test_x_candidates_fit_one_warp_per_row():
    for S in range(1, 9):
        for n in (16, 33, 100, 192):
            for m in autotune.candidates(n, S)[:-1]:
                assert math.ceil(n / m) * S <= 32


def test_shipped_cache_is_complete_and_valid():
    """The cache bench.py uses: every (edge bucket, substrate count) class present, each axis
    either whole lines or a chunk length the candidates allow for that class."""
    cache = autotune.load(autotune.default_cache_path())
    assert cache["precision"] == "fp32"
    for n in autotune.N_BUCKETS:
        for S in range(1, 9):
            m = cache["classes"][f"{n},{S}"]["m"]
            assert len(m) == 3
            for a, mm in enumerate(m):
                if mm == autotune.WHOLE:
                    continue
                allowed = autotune.candidates(n, S) if a == 0 else autotune.candidates(n)
                assert mm in allowed[:-1], (n, S, a, mm)
