"""Host-side admission of a serving loop by its device-memory budget: the
reservation a configuration needs is host arithmetic, and a server whose
reservation exceeds the budget is refused before any device call, so these
checks run without a GPU."""

import pytest

import paper_2601_12713_b300 as odp

OOM, CUDA, INVALID, UNSUPPORTED = -3, -2, -1, -7
SLOT_ALLOWANCE = 20 << 20  # granularity, beside the fingerprint scratch


def shape(**kw):
    d = dict(n_slots=4, max_events=1 << 20, max_batch_events=4096, max_producers=64)
    d.update(kw)
    return d


def test_reservation_grows_with_every_capacity():
    base = odp.server_bytes(**shape())
    assert odp.server_bytes(**shape(n_slots=5)) > base
    assert odp.server_bytes(**shape(max_events=1 << 21)) > base
    assert odp.server_bytes(**shape(max_batch_events=8192)) > base


def test_reservation_is_linear_in_slots():
    b = [odp.server_bytes(**shape(n_slots=k)) for k in (1, 2, 3, 8)]
    per_slot = b[1] - b[0]
    assert b[2] - b[1] == per_slot and b[3] - b[0] == 7 * per_slot
    # each slot holds at least its batch's event records, the allowance and
    # the fingerprint plan's tile arrays (44 bytes for each of 2^20 + n tiles)
    assert per_slot >= 4096 * 64 + SLOT_ALLOWANCE + 44 * ((1 << 20) + 4096)


def test_reservation_covers_the_resident_log():
    # 64-byte records of the resident log plus tables of twice its capacity
    small = odp.server_bytes(**shape(max_events=1 << 20))
    big = odp.server_bytes(**shape(max_events=1 << 22))
    assert big - small >= (3 << 20) * 64


def test_over_budget_is_refused_before_any_device_call():
    need = odp.server_bytes(**shape())
    with pytest.raises(odp.OdpError) as e:
        odp.Server(device_budget_bytes=need - 1, watermark_timeout_us=1000, **shape())
    assert e.value.status == OOM


def test_within_budget_reaches_the_device():
    import torch

    if torch.cuda.is_available():
        pytest.skip("on a GPU the server would be created")
    need = odp.server_bytes(**shape())
    # the budget admits it; without a GPU the first device call then fails
    with pytest.raises(odp.OdpError) as e:
        odp.Server(device_budget_bytes=need, watermark_timeout_us=1000, **shape())
    assert e.value.status == CUDA


@pytest.mark.parametrize("bad, status", [
    (dict(n_slots=0), INVALID),
    (dict(max_events=0), INVALID),
    (dict(max_batch_events=0), INVALID),
    (dict(max_producers=0), INVALID),
    (dict(max_events=(1 << 30) + 1), UNSUPPORTED),
    (dict(max_batch_events=(1 << 30) + 1), UNSUPPORTED),
])
def test_shape_errors(bad, status):
    with pytest.raises(odp.OdpError) as e:
        odp.server_bytes(**shape(**bad))
    assert e.value.status == status
    with pytest.raises(odp.OdpError) as e:
        odp.Server(device_budget_bytes=1 << 40, **shape(**bad))
    assert e.value.status == status
