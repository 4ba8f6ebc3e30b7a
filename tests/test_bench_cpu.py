"""Host-side bookkeeping of bench.py: the frame groups a decode runs as and
the kernel launches it claims (the JSON line's gpu_launches)."""
import argparse

import bench


def _bench():
    return bench


def _args(**kw):
    base = dict(launch_mode="graph", schedule="flooding", frame_groups=0)
    base.update(kw)
    return argparse.Namespace(**base)


def test_groups_follow_the_library_rule():
    b = _bench()
    assert b.groups_of(_args(), 16) == 2
    assert b.groups_of(_args(), 1) == 1
    assert b.groups_of(_args(frame_groups=3), 16) == 3
    assert b.groups_of(_args(frame_groups=9), 4) == 4
    assert b.groups_of(_args(schedule="layered"), 16) == 1
    assert b.groups_of(_args(schedule="layered", frame_groups=2), 16) == 2
    assert b.groups_of(_args(launch_mode="stream"), 16) == 1


def test_launch_count_of_a_grouped_decode():
    """Counted node by node for the graph the library builds: per step the
    LLR map, then per group an init, a loop of 4-pass trips of check pass,
    control step and posterior pass, and a final kernel."""
    b = _bench()
    # two groups whose slowest frames stopped after passes 501 and 7:
    # trips of 4 passes -> 126 and 2 trips
    expect = 1 + 2 * (1 + 1) + (126 * 4 * 3) + (2 * 4 * 3)
    assert b.launch_count([501, 7], 3, 4) == expect
    # one chain, stream launches: every pass enqueued, no trips
    assert b.launch_count([501], 3, 1) == 1 + 2 + 501 * 3
    # layered with 49 row groups: 2 + 2 * 49 kernels per pass, one per trip
    assert b.launch_count([10, 12], 2 + 2 * 49, 1) == 1 + 4 + (10 + 12) * 100
