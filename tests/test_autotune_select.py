"""The autotuner's choice from its timing table (host logic, no GPU): the fastest accepted
candidate, the earliest of equal times, and the fastest accepted tensor-core candidate when it
is within 1 % of that."""
from paper_2309_15642_gb300.autotune import TENSOR_SLACK, candidates, select

REF = dict(persistent=0, tol=1e-9, floor_rel=1e-11, tol32=1e-6, floor32=2e-7)


def _row(ms, accepted=True, reference=False, **cand):
    return dict(cand, ms_per_step=ms, max_dz=0.0, max_dz_reference=None, accepted=accepted,
                reference=reference)


def test_fastest_accepted_candidate_wins():
    table = [_row(30.0, reference=True, **REF),
             _row(25.0, persistent=5, tensor=False, floor_rel=1e-7),
             _row(20.0, accepted=False, persistent=6, tensor=False, floor_rel=1e-7),
             _row(None, accepted=False, persistent=3, tensor=True),
             _row(22.0, persistent=6, tensor=False, floor_rel=7e-8)]
    ms, cand = select(table)
    assert ms == 22.0 and cand == dict(persistent=6, tensor=False, floor_rel=7e-8)


def test_tensor_cores_preferred_within_slack_only():
    cuda = _row(22.0, persistent=6, tensor=False)
    near = _row(22.0 * (1 + TENSOR_SLACK) * 0.999, persistent=6, tensor=True)
    far = _row(22.0 * (1 + TENSOR_SLACK) * 1.01, persistent=5, tensor=True)
    assert select([_row(30.0, reference=True, **REF), cuda, near])[1]["tensor"] is True
    assert select([_row(30.0, reference=True, **REF), cuda, far])[1]["tensor"] is False
    # a rejected tensor-core row is never chosen
    bad = dict(near, accepted=False)
    assert select([_row(30.0, reference=True, **REF), cuda, bad])[1]["tensor"] is False


def test_reference_kept_when_nothing_is_faster_and_ties_keep_the_earlier_row():
    ref = _row(20.0, reference=True, **REF)
    ms, cand = select([ref, _row(21.0, persistent=5, tensor=False)])
    assert ms == 20.0 and cand == REF
    a, b = _row(19.0, persistent=4, tensor=False), _row(19.0, persistent=5, tensor=False)
    assert select([ref, a, b])[1]["persistent"] == 4


def test_candidate_grid():
    mixed = candidates("mixed", 32)
    assert {c["persistent"] for c in mixed} == {0, 1, 2, 3, 4, 5, 6}
    assert {c["tensor"] for c in mixed} == {False, True}
    assert all(c["floor_rel"] <= 0.7 * c["floor32"] * (1 + 1e-9) for c in mixed)
    assert {c["tensor"] for c in candidates("mixed", 16)} == {False}
    assert candidates("c128", 32) == [dict(persistent=p) for p in range(7)]
