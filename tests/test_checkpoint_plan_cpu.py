"""The gradient's checkpoint planner (host only) against a plain recount of the merged DP's
layers.  The layer sizes and per-layer work are recomputed here from the definition of the
state space (interaction masks with vertex 0 visited, heads and reachable endpoints), not
taken from the library, and every checkpoint set of the search space is evaluated by brute
force: the planner's answer must be an optimum of storage within the budget."""
import itertools

import pytest

from paper_2507_12349_b300 import binding as B


def _row_vmask(A, ones, h):
    if h == 0:
        if ones & 1:
            return 1 if A == 1 else (A & ~1)
        return A
    v = A & ~1
    if ones & ((1 << h) - 1):
        v &= ~(1 << h)
    return v


def layer_counts(n):
    """Slots (|H| x |A| per mask) and sweep work (reachable endpoints x (extensions + close))
    per layer l = number of visited points."""
    full = (1 << n) - 1
    slots = [0] * (2 * n + 2)
    work = [0] * (2 * n + 2)
    for code in range(3 ** n):
        x, A, Bf, layer = code, 0, 0, 0
        for i in range(n):
            d = x % 3
            x //= 3
            A |= (d >= 1) << i
            Bf |= (d == 2) << i
            layer += d
        if not A & 1:
            continue
        ones = A & ~Bf
        H = 1 if ones & 1 else Bf
        nJ = bin(full & ~Bf).count("1")
        close = 1 if (ones or Bf == full) else 0
        slots[layer] += bin(H).count("1") * bin(A).count("1")
        for h in range(n):
            if H >> h & 1:
                work[layer] += bin(_row_vmask(A, ones, h)).count("1") * (nJ + close)
    return slots, work


def evaluate(n, slots, work, cks):
    starts = [1] + sorted(cks)
    ends = starts[1:] + [2 * n + 1]
    store = sum(slots[a] for a in starts) + max(sum(slots[a + 1:b]) for a, b in zip(starts, ends))
    rec = sum(sum(work[a:b - 1]) for a, b in list(zip(starts, ends))[:-1])
    return store, rec


@pytest.mark.parametrize("n", [3, 5, 6])
def test_planner_is_optimal_for_every_budget(n):
    slots, work = layer_counts(n)
    cand = [evaluate(n, slots, work, c) + (c,) for k in range(0, 8)
            for c in itertools.combinations(range(2, 2 * n + 1), k)]
    full = sum(slots[1:2 * n + 1])
    assert evaluate(n, slots, work, ())[0] == full
    least = min(c[0] for c in cand)
    for budget in sorted({c[0] for c in cand}) + [full + 7]:
        mask, store, rec = B.cos_grad_checkpoint_plan(n, budget)
        cks = tuple(l for l in range(2, 2 * n + 1) if mask >> l & 1)
        assert mask & 3 == 0 and mask >> (2 * n + 1) == 0
        assert (store, rec) == evaluate(n, slots, work, cks)        # the layout the kernel uses
        assert store <= budget
        assert rec == min(c[1] for c in cand if c[0] <= budget)     # least recomputation that fits
    mask, store, rec = B.cos_grad_checkpoint_plan(n, 0)
    assert store == least
    assert B.cos_grad_checkpoint_plan(n, full)[0] == 0               # everything fits: no checkpoints


def test_planner_rejects_budgets_below_the_least_storage():
    least = B.cos_grad_checkpoint_plan(8, 0)[1]
    with pytest.raises(B.CosError):
        B.cos_grad_checkpoint_plan(8, least - 1)
    with pytest.raises(B.CosError):
        B.cos_grad_checkpoint_plan(13, 0)


def test_order_12_fits_in_about_70_percent():
    """The memory-bound order: 70 % of the full storage costs about a quarter of one forward
    sweep in recomputation (layer counts of the library's own structure)."""
    s = B.cos_structure(12)
    mask, store, rec = B.cos_grad_checkpoint_plan(12, int(0.7 * s.slots))
    assert store <= 0.7 * s.slots and mask != 0
    assert rec < 0.3 * (s.fma_ext + s.fma_close)
