"""Host logic of the batch autotuner: candidate grids and the choice."""
from paper_1909_01589_gb300.batch import candidate_grids, candidate_plans, choose


def test_candidates_respect_limits_and_proportions():
    defaults = [608, 608, 456, 304, 608]
    work = [0.2, 1.5, 6.0, 30.0, 2.0]
    need = [2048, 2048, 2048, 2048, 2048]
    cands = candidate_grids(defaults, work, need)
    names = [c[0] for c in cands]
    assert names[0] == "default" and cands[0][1] == defaults
    for _, b in cands:
        assert all(1 <= x <= min(d, m) for x, d, m in zip(b, defaults, need))
    prop = dict(cands)["proportional x1"]
    # more work, larger share of its own default grid
    shares = [b / d for b, d in zip(prop, defaults)]
    order = sorted(range(5), key=lambda i: work[i])
    assert [shares[i] for i in order] == sorted(shares)
    # candidates are distinct
    assert len({tuple(b) for _, b in cands}) == len(cands)


def test_small_populations_cap_the_grid():
    cands = candidate_grids([608, 608], [1.0, 1.0], [3, 600])
    for _, b in cands:
        assert b[0] <= 3 and b[1] <= 600


def test_single_system_has_only_the_default():
    assert candidate_grids([608], [1.0], [100]) == [("default", [100])]


def test_plans_cover_concurrent_serial_and_split():
    defaults = [608, 608, 304]
    work = [2.0, 10.0, 50.0]
    need = [4096, 4096, 4096]
    plans = candidate_plans(defaults, work, need)
    names = [p[0] for p in plans]
    assert names[0] == "concurrent default"
    serial = dict((p[0], p[1]) for p in plans)["serial"]
    assert sorted(serial) == [0, 1, 2] and serial[2] == 0 and serial[0] == 2  # heaviest first
    split = [p for p in plans if p[0].startswith("heaviest alone")]
    assert split and all(p[1] == [1, 1, 0] for p in split)
    for _, groups, blocks, carve, pipe in plans:
        assert len(groups) == 3 and all(1 <= b <= d for b, d in zip(blocks, defaults)) and carve in (-1, 100)
        assert pipe in (0, 1)
    assert any(p[3] == 100 for p in plans) and any(p[3] == -1 for p in plans)
    piped = dict((p[0], p) for p in plans if p[4] == 1)
    assert piped["pipelined, heaviest first"][1] == serial
    assert piped["pipelined, lightest first"][1] == [2 - r for r in serial]


def test_choose_takes_the_fastest():
    t = [("a", [0, 0], [608, 608], -1, 0, 10.0), ("b", [0, 1], [100, 500], 100, 1, 7.5),
         ("c", [0, 0], [304, 304], -1, 0, 8.0)]
    assert choose(t) == ("b", [0, 1], [100, 500], 100, 1, 7.5)
