"""Host logic of the launch-shape autotuner (no GPU: the timed function is synthetic)."""
import os

from paper_2112_00087_gb300 import autotune as at


def fake_solve():
    # separable cost with its minimum at 3 blocks/SM, 2,048-row tiles, 2 tiles per block,
    # prefetch 0, 4 chunks
    b = int(os.environ["HELM_PERSIST_BLOCKS_PER_SM"])
    t = int(os.environ["HELM_TILE_ROWS"])
    g = int(os.environ["HELM_TILES_PER_BLOCK"])
    p = int(os.environ["HELM_PREFETCH"])
    c = int(os.environ["HELM_PF_CHUNKS"])
    return 1.0 + 0.3 * abs(b - 3) + 0.1 * abs(t - 2048) / 2048 + 0.04 * abs(g - 2) + 0.05 * p + 0.02 * abs(c - 4)


def test_coordinate_descent_finds_the_minimum_and_restores_the_environment():
    before = {k: os.environ.get(k) for k in at.SPACE}
    best, log = at.autotune(fake_solve)
    assert best == {"HELM_PERSIST_BLOCKS_PER_SM": 3, "HELM_TILE_ROWS": 2048, "HELM_TILES_PER_BLOCK": 2,
                    "HELM_PREFETCH": 0, "HELM_PF_CHUNKS": 4}
    assert {k: os.environ.get(k) for k in at.SPACE} == before
    keys = [tuple(sorted(c.items())) for c, _ in log]
    assert len(keys) == len(set(keys))  # every setting timed once
    best_t = [t for c, t in log if c == best][0]
    assert best_t == min(t for _, t in log)


def test_apply_installs_the_setting():
    saved = {k: os.environ.get(k) for k in at.SPACE}
    try:
        at.apply({"HELM_PREFETCH": 2, "HELM_TILE_ROWS": 8192})
        assert os.environ["HELM_PREFETCH"] == "2" and os.environ["HELM_TILE_ROWS"] == "8192"
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_repetitions_take_the_minimum():
    calls = []

    def noisy():
        calls.append(1)
        return 2.0 if len(calls) % 2 else 1.0

    best, log = at.autotune(noisy, space={"HELM_PREFETCH": (0, 1)}, start={"HELM_PREFETCH": 1}, reps=2)
    assert all(t == 1.0 for _, t in log) and len(calls) == 4


def test_gains_below_the_threshold_keep_the_current_value():
    # a knob that changes nothing (times equal to 0.03 %) is left at its start value
    times = {1: 6.7760, 2: 6.7779, 4: 6.7781}

    def run():
        return times[int(os.environ["HELM_TILES_PER_BLOCK"])]

    best, _ = at.autotune(run, space={"HELM_TILES_PER_BLOCK": (1, 2, 4)}, start={"HELM_TILES_PER_BLOCK": 2})
    assert best == {"HELM_TILES_PER_BLOCK": 2}
    best, _ = at.autotune(run, space={"HELM_TILES_PER_BLOCK": (1, 2, 4)}, start={"HELM_TILES_PER_BLOCK": 2},
                          min_gain=0.0)
    assert best == {"HELM_TILES_PER_BLOCK": 1}
