"""The shared-memory bank model that picks the FFT exchange-plane row padding."""
from paper_1202_3424_gb300 import bank_model as bm


def test_wavefront_counts_of_textbook_patterns():
    # consecutive 8-byte elements: one wavefront per half-warp
    assert bm.wavefronts([8 * i for i in range(32)]) == 2
    # every thread on the same element: broadcast
    assert bm.wavefronts([0] * 32) == 2
    # a 128-byte stride puts all 16 threads of a phase on banks 0-1 with distinct words
    assert bm.wavefronts([128 * i for i in range(32)]) == 32
    # a 64-byte stride: eight threads on each of two bank pairs -> 8 per phase
    assert bm.wavefronts([64 * i for i in range(32)]) == 16
    # a 136-byte stride (17 elements): conflict-free
    assert bm.wavefronts([136 * i for i in range(32)]) == 2


def test_exchange_positions_cover_the_pencil_once_per_instruction_set():
    # every store set of one stage writes each position exactly once
    plans = bm.read_plans()
    for L, (NT, rad) in plans["Plan"].items():
        seen = []
        for pos in bm.exchange_positions(L, NT, rad, -1):
            seen.extend(pos)
        n_ex = len(rad) - 1
        assert len(seen) == 2 * n_ex * L
        assert sorted(seen) == sorted(list(range(L)) * 2 * n_ex)


def test_padded_rows_are_distinct_and_fit_the_plane():
    for (L, NT, TP), sh in bm.read_table().items():
        rows = [bm.padded_row(p, sh) for p in range(L)]
        assert len(set(rows)) == L, (L, NT, TP)
        # the kernels size a plane as L + ((L - 1) >> S) rows
        assert max(rows) + 1 == L + ((L - 1) >> sh)


def test_header_table_is_the_models_choice():
    want = {k: v[0] for k, v in bm.table().items() if v[0] != 0}
    assert bm.read_table() == want


def test_padding_removes_the_narrow_tile_conflicts():
    NT, rad = bm.read_plans()["Plan"][512]
    a, i = bm.cost(512, NT, rad, 4)
    assert a / i > 1.5
    a, i = bm.cost(512, NT, rad, 4, 3)
    assert a == i


def test_warp_plans_are_valid_stockham_schedules():
    """Every warp-local plan fits a warp, and every radix divides the points
    per lane with NT dividing L/R (the stage layout's requirements)."""
    for (L, V), (NT, rad) in bm.read_warp_plans().items():
        E = L // NT
        assert NT <= 32 and 32 % NT == 0 and L % NT == 0, (L, V)
        prod = 1
        for R in rad:
            prod *= R
            assert E % R == 0 and (L // R) % NT == 0, (L, V, R)
        assert prod == L and rad[0] % 2 == 0, (L, V)


def test_warp_swizzle_is_a_permutation_within_the_plane():
    for key in range(1, 7):
        for L in (64, 96, 128, 192, 256, 384, 512):
            slots = {bm.warp_swizzle(p, key) for p in range(L)}
            assert slots == set(range(L)), (L, key)


def test_warp_header_tables_are_the_models_choice():
    keys, pads, costs = bm.warp_table()
    have, have_pads = bm.read_warp_table()
    assert have == {k: v for k, v in keys.items() if v}
    assert have_pads == pads
    # the hot lengths reach the ideal wavefront count within 15 %
    for (L, NT), (c, plain) in costs.items():
        if L >= 64:
            assert c <= 1.15, (L, NT, c)
