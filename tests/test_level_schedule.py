"""The ticket list of the one-launch level kernel (host logic, no GPU): every
field of every patch size is solved exactly once, a 256^2 field takes a whole
cluster ticket, the other sizes fill CTA tasks of 65 536 cells, and the two
schedules order the tickets as stated."""
import math

import numpy as np
import pytest

CELLS = {32: 16, 64: 4, 128: 1}           # fields per CTA task
CODE = {32: 0, 64: 1, 128: 2, 256: 3}
SIZE = {v: k for k, v in CODE.items()}


def _decode(code):
    return SIZE[int(code) >> 56], int(code) & ((1 << 56) - 1)


def _fields_of(tickets, counts):
    """Each (size, field item) the tickets hand out, and each ticket's kind."""
    got = {n: [] for n in counts}
    kinds = []
    for t in tickets:
        codes = [int(c) for c in t]
        if codes[0] >= 0 and _decode(codes[0])[0] == 256:
            assert codes == [codes[0]] * 4, t       # the whole cluster on one field
            got[256].append(_decode(codes[0])[1])
            kinds.append("big")
            continue
        for c in codes:
            if c < 0:
                continue
            n, it = _decode(c)
            assert n != 256, t
            assert it % CELLS[n] == 0, (n, it)
            got[n].extend(range(it, min(it + CELLS[n], 2 * counts[n])))
        kinds.append("cta")
    return got, kinds


@pytest.mark.parametrize("sizes,counts", [
    ([64, 128, 256], [3166, 60090, 2280]),       # the 4th octave level of the continuous spectrum
    ([32, 64], [24538, 40998]),                  # the 5th
    ([32, 64, 128, 256], [7, 5, 3, 2]),
    ([256, 32], [1, 1]),
    ([128, 64], [1, 9]),
])
@pytest.mark.parametrize("schedule", [0, 1])
def test_every_field_once_and_ticket_shapes(sizes, counts, schedule):
    import paper_1510_00451_gb300 as m
    t = m.level_schedule(sizes, counts, schedule)
    cnt = dict(zip(sizes, counts))
    got, kinds = _fields_of(t, cnt)
    for n in sizes:
        assert sorted(got[n]) == list(range(2 * cnt[n])), n
    n_cta = sum(math.ceil(2 * cnt[n] / CELLS[n]) for n in sizes if n != 256)
    nb = 2 * cnt.get(256, 0)
    assert len(t) == nb + math.ceil(n_cta / 4)
    # CTA tasks: larger patches first, padding only at the end
    cta = [int(c) for t_, k in zip(t, kinds) if k == "cta" for c in t_]
    real = [c for c in cta if c >= 0]
    assert cta[:len(real)] == real
    order = [_decode(c)[0] for c in real]
    assert order == sorted(order, reverse=True)
    big_pos = [i for i, k in enumerate(kinds) if k == "big"]
    if schedule == 0:
        assert big_pos == list(range(nb))
    elif nb:
        # the k-th 256^2 ticket sits where k / nb of the tickets lie before it
        nt = len(t)
        for k, p in enumerate(big_pos):
            assert abs(p - k * nt / nb) <= 1.0, (k, p, nt, nb)


def test_schedule_rejects_bad_arguments():
    import ctypes
    import paper_1510_00451_gb300 as m
    L = m.lib()
    n = np.array([64, 48], np.int32)
    c = np.array([3, 3], np.int64)
    nt = ctypes.c_int64()
    # 48 has no task shape; a size twice; no classes; an unknown schedule
    assert L.mlsd_level_schedule(n.ctypes.data, c.ctypes.data, 2, 0, 0, None, ctypes.byref(nt)) == -1
    n2 = np.array([64, 64], np.int32)
    assert L.mlsd_level_schedule(n2.ctypes.data, c.ctypes.data, 2, 0, 0, None, ctypes.byref(nt)) == -1
    assert L.mlsd_level_schedule(n.ctypes.data, c.ctypes.data, 0, 0, 0, None, ctypes.byref(nt)) == -1
    n3 = np.array([64, 128], np.int32)
    assert L.mlsd_level_schedule(n3.ctypes.data, c.ctypes.data, 2, 2, 0, None, ctypes.byref(nt)) == -1
    # too small a capacity: the count is still reported
    assert L.mlsd_level_schedule(n3.ctypes.data, c.ctypes.data, 2, 0, 0, None, ctypes.byref(nt)) == -1
    assert nt.value == math.ceil((math.ceil(6 / 4) + 6) / 4)
