"""The serving layer's shared-budget admission policy (one step, as the
server applies it between chunks), evaluated on described states without a
GPU through amto_admission_step: a count whose queue exceeds its free slots
doubles its capacity, from unclaimed budget and from other counts' free
slots; idle counts shrink to max(min(8, fair), next power of two >= resident),
counts with a queue keep their fair share; changes under a quarter of a
capacity are not made; the budget is never exceeded."""
import pytest

PER = (1000, 3000)  # bytes per instance of two counts


@pytest.fixture(scope="module")
def amto():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_04240_b300 import amto as A
    A.load()
    return A


def step(amto, slots, active, queued, fair, cap, per=PER, budget=None):
    if budget is None:
        budget = sum(f * p for f, p in zip(fair, per))
    out = amto.admission_step(slots, active, queued, fair, cap, per, budget)
    used = sum(s * p for s, p in zip(out, per))
    assert used <= max(budget, sum(s * p for s, p in zip(slots, per)))
    return out


def test_flooded_count_grows_from_an_idle_one(amto):
    # count 1 (3000 B) full with 50 queued; count 0 (1000 B) idle with 40 slots; the budget
    # is all used: count 0 gives its free slots down to 8 (32000 B), which buys count 1 ten
    # more slots (its target, 32 = its largest capacity, needs 36000 B)
    out = step(amto, [40, 20], [0, 20], [0, 50], [40, 20], [64, 32])
    assert out == [8, 30]


def test_budget_is_never_exceeded(amto):
    per = (1000, 3000)
    budget = 40 * 1000 + 20 * 3000
    out = amto.admission_step([40, 20], [0, 20], [0, 50], [40, 20], [64, 32], per, budget)
    assert out[0] * 1000 + out[1] * 3000 <= budget
    assert out[1] > 20 and out[0] < 40


def test_queued_count_keeps_its_fair_share(amto):
    # both counts have queues: the one above its fair share is not a donor below it
    budget = 40 * 1000 + 20 * 3000
    out = amto.admission_step([40, 20], [40, 20], [5, 50], [40, 20], [64, 32], PER, budget)
    assert out[0] == 40 and out[1] == 20


def test_resident_requests_bound_the_shrink(amto):
    # the idle count holds 20 resident requests: it shrinks to 32 at most (power of two)
    budget = 64 * 1000 + 10 * 3000
    out = amto.admission_step([64, 10], [20, 10], [0, 40], [32, 10], [64, 64], PER, budget)
    assert out[0] == 32
    assert out[1] > 10
    assert out[0] * 1000 + out[1] * 3000 <= budget


def test_small_changes_are_not_made(amto):
    # free budget for one more slot only: below a quarter of the capacity, no change
    budget = 40 * 1000 + 20 * 3000 + 3000
    out = amto.admission_step([40, 20], [40, 20], [1, 5], [40, 20], [64, 64], PER, budget)
    assert out == [40, 20]


def test_nothing_queued_nothing_changes(amto):
    out = amto.admission_step([8, 16], [3, 16], [0, 0], [8, 16], [64, 64], PER, 10 ** 6)
    assert out == [8, 16]


def test_one_count_grows_per_step(amto):
    per = (1000, 1000, 1000)
    out = amto.admission_step([8, 8, 8], [8, 8, 8], [30, 20, 0], [8, 8, 8], [64, 64, 64], per,
                              10 ** 6)
    # the largest unmet queue only; at least the next power of two above resident + queued
    assert out == [64, 8, 8]


def test_rejects_bad_descriptions(amto):
    with pytest.raises(amto.AmtoError):
        amto.admission_step([8], [9], [0], [8], [8], (1000,), 10 ** 6)   # active > slots
    with pytest.raises(amto.AmtoError):
        amto.admission_step([8], [0], [0], [8], [4], (1000,), 10 ** 6)   # cap < slots
