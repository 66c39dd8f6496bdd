"""The bench's block schedule on CPU: whatever --steps and --warmup the
caller gives, no MD system runs past the workload's 100 MD steps (the seeded
model barely holds the lattice, so a system run much longer drifts into close
contacts), every requested block runs exactly once, and the timed system that
is kept for the accuracy check is the last one."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeSystem:
    def __init__(self, k):
        self.id = k
        self.md_steps = 0
        self.alive = True


def simulate(nblocks, keep_last):
    made, ran = [], []

    def create():
        s = FakeSystem(len(made))
        made.append(s)
        return s

    def run(s, nb):
        assert s.alive
        s.md_steps += bench.MD_PER_STEP * nb
        ran.append(nb)

    def destroy(s):
        assert s.alive
        s.alive = False

    last = bench.run_schedule(create, run, destroy, nblocks, keep_last=keep_last)
    return made, ran, last


@pytest.mark.parametrize("nblocks", [0, 1, 3, 5, 9, 10, 11, 20, 25, 37, 100])
@pytest.mark.parametrize("keep_last", [False, True])
def test_no_system_past_100_md_steps(nblocks, keep_last):
    made, ran, last = simulate(nblocks, keep_last)
    assert sum(ran) == nblocks
    assert all(s.md_steps <= 100 for s in made)
    assert len(made) == -(-nblocks // bench.MAX_BLOCKS_PER_SYSTEM)
    if keep_last and nblocks:
        assert last is made[-1] and last.alive
        assert all(not s.alive for s in made[:-1])
    else:
        assert last is None and all(not s.alive for s in made)


def test_driver_counts():
    # the round-end command: --steps 20 --warmup 5 (warm-up on systems of its own)
    for n in (5, 20):
        made, ran, _ = simulate(n, keep_last=True)
        assert max(s.md_steps for s in made) <= 100
    assert bench.block_segments(20) == [10, 10]
    assert bench.block_segments(5) == [5]
    assert bench.block_segments(0) == []
    with pytest.raises(ValueError):
        bench.block_segments(-1)
