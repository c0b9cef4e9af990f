"""The autotuner's search on the host: coordinate descent over tile size,
render schedule, forward and backward staging depth, with a synthetic cost in
place of GPU timing (the library is loaded for its config struct only)."""
import pytest

from paper_2506_05558_gb300 import autotune, gs


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_05558_gb300 import build
    build.build()


def run_with_cost(monkeypatch, cost):
    seen = []

    def fake(g, cams, sizes, targets, cfg, steps=3, device="cuda"):
        key = (cfg.tile, cfg.fwd_batch, cfg.bwd_batch, cfg.schedule)
        seen.append(key)
        return cost(*key)

    monkeypatch.setattr(autotune, "time_config", fake)
    cfg, table = autotune.tune(None, None, None, None, gs.config(), steps=1, device="cpu")
    return (cfg.tile, cfg.fwd_batch, cfg.bwd_batch, cfg.schedule), table, seen


def test_descends_each_coordinate_in_order(monkeypatch):
    # separable cost: tile 16 best, persistent schedule better, fwd 128, bwd 64
    def cost(tile, fb, bb, sched):
        c = {8: 14.0, 16: 11.0, 32: 22.0}[tile]
        c -= 0.3 if sched == 1 else 0.0
        c -= {0: 0.0, 64: 0.05, 128: 0.2, 256: 0.1}.get(fb, 0.0)
        c -= {0: 0.0, 32: -0.5, 64: 0.25, 128: 0.1}.get(bb, 0.0)
        return c

    best, table, seen = run_with_cost(monkeypatch, cost)
    assert best == (16, 128, 64, 1)
    # tiles first, then the schedules (persistent, ordered grid) at the best tile, then fwd depths,
    # then bwd depths
    assert seen[:3] == [(8, 0, 0, 0), (16, 0, 0, 0), (32, 0, 0, 0)]
    assert seen[3:5] == [(16, 0, 0, 1), (16, 0, 0, 2)]
    assert seen[5:8] == [(16, fb, 0, 1) for fb in autotune.FWD_BATCHES[16]]
    assert seen[8:] == [(16, 128, bb, 1) for bb in autotune.BWD_BATCHES[16]]
    assert len(table) == len(seen) and all(len(row) == 5 for row in table)


def test_failed_configs_are_never_chosen(monkeypatch):
    # a configuration that overflows (time_config returns inf) loses to any finite one
    def cost(tile, fb, bb, sched):
        if tile == 8 or bb == 32:
            return float("inf")
        return 10.0 + (0.5 if tile == 32 else 0.0) - (0.1 if fb == 256 else 0.0)

    best, _, _ = run_with_cost(monkeypatch, cost)
    assert best[0] == 16 and best[2] != 32 and best[1] == 256


def test_ordered_grid_schedule_chosen_when_fastest(monkeypatch):
    def cost(tile, fb, bb, sched):
        return {8: 14.0, 16: 11.0, 32: 22.0}[tile] - {0: 0.0, 1: 0.1, 2: 0.2}[sched]

    best, _, _ = run_with_cost(monkeypatch, cost)
    assert best == (16, 0, 0, 2)


def test_defaults_kept_when_nothing_improves(monkeypatch):
    best, _, _ = run_with_cost(monkeypatch, lambda *k: 5.0)
    assert best == (8, 0, 0, 0)  # first tile tried, default depths, grid schedule
