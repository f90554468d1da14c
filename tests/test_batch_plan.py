"""The batched work split (swp_batch_plan, host only, no GPU): every system is
advanced exactly once by a group of distinct blocks, a block's group share
comes first so that group members start together, and the balanced plan keeps
the largest per-block load near the mean on the batched workload's size mix
(256 systems, log-uniform 1k-32k particles, 152 blocks)."""
import numpy as np
import pytest

B = 152


@pytest.fixture(scope="module")
def A():
    from paper_1912_08569_gb300 import _abi
    from paper_1912_08569_gb300.build import build

    build()
    _abi.load_library()
    return _abi


def _check_plan(w, ofs, items, n_blocks, max_group, min_part, balanced):
    """Structural invariants; returns the per-block loads."""
    m = len(w)
    assert len(ofs) == n_blocks + 1 and ofs[0] == 0 and ofs[-1] == len(items)
    assert np.all(np.diff(ofs) >= 0)
    assert len(items) <= m + n_blocks
    block_of = np.repeat(np.arange(n_blocks), np.diff(ofs))
    ranks = {}
    for (r, k, g, z), b in zip(items, block_of):
        assert 0 <= r < m and z == 0 and 1 <= g <= max_group and 0 <= k < g
        ranks.setdefault(r, []).append((k, g, b))
    assert sorted(ranks) == list(range(m)), "every system exactly once"
    load = np.zeros(n_blocks)
    for r, lst in ranks.items():
        g = lst[0][1]
        assert all(x[1] == g for x in lst)
        assert sorted(x[0] for x in lst) == list(range(g))
        assert len({x[2] for x in lst}) == g, "a group's members are distinct blocks"
        if g > 1 and balanced:
            assert w[r] // g >= min_part
        for _, _, b in lst:
            load[b] += max(w[r], 1) / g
    for b in range(n_blocks):
        its = items[ofs[b]:ofs[b + 1]]
        multi = [i for i, it in enumerate(its) if it[2] > 1]
        if balanced:
            # at most one group share per block, and it runs first
            assert multi in ([], [0])
        else:
            assert not multi or len(its) == 1
    return load


def _sizes(seed):
    from paper_1912_08569_gb300 import inputs

    return [p[0] for p in inputs.batch_params(256, seed=seed)]


def test_batch_params_match_the_workload():
    from paper_1912_08569_gb300 import inputs

    wls = inputs.batch_workload(6, seed=3, n_min=100, n_max=400)
    ps = inputs.batch_params(6, seed=3, n_min=100, n_max=400)
    assert [wl["n"] for wl in wls] == [p[0] for p in ps]
    assert [wl["kT"] for wl in wls] == [p[2] for p in ps]


@pytest.mark.parametrize("seed", [1, 2, 7])
def test_balanced_plan_on_the_batched_size_mix(A, seed):
    w = _sizes(seed)
    ofs, items = A.swp_batch_plan(w, B, 0.0, 304, 1024)
    load = _check_plan(w, ofs, items, B, 304, 1024, True)
    mean = sum(w) / B
    assert load.max() <= 1.15 * mean, load.max() / mean
    # no worse than any threshold plan
    for split in (0.5, 1.0, 2.0, 1e9):
        o2, i2 = A.swp_batch_plan(w, B, split, 304, 1024)
        l2 = _check_plan(w, o2, i2, B, 304, 1024, False)
        assert load.max() <= l2.max() + 1e-9, split
    # deterministic
    o3, i3 = A.swp_batch_plan(w, B, 0.0, 304, 1024)
    assert np.array_equal(ofs, o3) and np.array_equal(items, i3)


@pytest.mark.parametrize("w,n_blocks,min_part", [
    ([4100, 3000, 2200, 900, 300], B, 1024),   # a few small systems: shares of at least min_part
    ([1], 8, 256),
    ([0, 0, 5], 4, 256),
    ([100000], B, 1024),                       # one large system over many blocks
    ([5000] * 300, B, 1024),                    # more systems than blocks
    ([30000, 20, 20, 20], 4, 256),
    (list(np.random.default_rng(3).integers(1, 50000, size=1000)), B, 512),
])
def test_plans_are_valid(A, w, n_blocks, min_part):
    w = [int(x) for x in w]
    for split in (0.0, 0.5, 1.0, 1e9):
        try:
            ofs, items = A.swp_batch_plan(w, n_blocks, split, 304, min_part)
        except A.SwpError:
            # only the threshold plan may give up (more large systems than blocks)
            assert split > 0.0
            continue
        load = _check_plan(w, ofs, items, n_blocks, 304, min_part, split == 0.0)
        assert load.max() >= sum(max(x, 1) for x in w) / n_blocks - 1e-9


def test_balanced_plan_is_optimal_on_tiny_cases(A):
    """Against the best assignment without groups (brute force): the balanced
    plan's largest load is within the longest-processing-time rule's bound
    (4/3 - 1/(3B)) of it, and never above it where groups can help."""
    import itertools

    rng = np.random.default_rng(11)
    for _ in range(40):
        m, nb = int(rng.integers(1, 7)), int(rng.integers(1, 4))
        w = [int(x) for x in rng.integers(1, 100, size=m)]
        best = min(max(sum(w[r] for r in range(m) if a[r] == b) for b in range(nb))
                   for a in itertools.product(range(nb), repeat=m))
        ofs, items = A.swp_batch_plan(w, nb, 0.0, 304, 1)
        load = _check_plan(w, ofs, items, nb, 304, 1, True)
        assert load.max() <= (4.0 / 3.0 - 1.0 / (3 * nb)) * best * (1 + 1e-5), (w, nb, load.max(), best)


def test_plan_rejects_bad_arguments(A):
    with pytest.raises(A.SwpError):
        A.swp_batch_plan([10, 20], 0, 0.0, 304, 1024)
    with pytest.raises(A.SwpError):
        A.swp_batch_plan([10, -1], 4, 0.0, 304, 1024)
    with pytest.raises(A.SwpError):
        A.swp_batch_plan([10, 20], 4, -1.0, 304, 1024)

