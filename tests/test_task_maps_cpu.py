"""Host replay of the row-task maps of the split Chebyshev kernels (k_yanalysis, k_ysynth).

The per-mode Chebyshev analysis and synthesis of the descent step (§4, the transforms inside
steps 1 and 3) fold each transform by the parity of T_n: a class of rows (even or odd
coefficients; values at y_j and y_{N-j}) is computed two rows per lane.  In FP64 the middle
row of a class with an odd number of rows runs as its own tasks after the pairs, where its
pair with a dead row would have started a warp of its own.  These tests
restate the kernels' task arithmetic on the host and check, for every grid the library accepts
(ny odd, 9..129), every group size and every mode tile, that
- every output (row, column) is written exactly once,
- every table row read is inside its table,
- no warp mixes pair tasks and single-row tasks (their loops differ).
They need no GPU and do not use the oracle."""
import itertools

import pytest


def col_pad(n_inst):
    sp = 2
    while sp < 2 * n_inst:
        sp <<= 1
    return sp


def round_up(a, b):
    return (a + b - 1) // b * b


def _warps_uniform(ntask, kind_of):
    for w in range(0, ntask, 32):
        if len({kind_of(t) for t in range(w, min(w + 32, ntask))}) != 1:
            return False
    return True


def _issued(ntask, fma_of):
    """FP64 multiply-add warp-instructions of a CTA: per warp, its lanes' count (uniform)."""
    return sum(fma_of(w) for w in range(0, ntask, 32))


def synthesis_tasks(N, n_inst, mt, fp64):
    """Outputs written by one k_ysynth CTA, [(y index, mode, instance, part)], and its issued
    FP64 multiply-adds (a pair: both rows' even and odd chains; a single row: its two)."""
    H, half = N // 2 + 1, N // 2
    SP = col_pad(n_inst)
    SPt = SP * mt
    RW = 32 // SPt
    hJ = (H + 1) // 2
    lone = fp64 and H % 2 == 1 and (hJ - 1) % RW == 0
    npair = hJ - (1 if lone else 0)
    PT = round_up(npair, RW) * SPt
    ntask = PT + (SPt if lone else 0)
    assert PT % 32 == 0 and _warps_uniform(ntask, lambda t: t >= PT)
    out = []
    for t in range(ntask):
        if t >= PT:
            sc, j = t - PT, hJ - 1
            assert 0 <= j < H
            mm = sc // SP
            i, part = (sc - mm * SP) >> 1, sc & 1
            if i >= n_inst or mm >= mt:
                continue
            out += [(j, mm, i, part)] + ([(N - j, mm, i, part)] if j < half else [])
            continue
        sc, j0 = t % SPt, t // SPt
        j1, mm = j0 + hJ, sc // SP
        v0 = j0 < npair
        v1 = v0 and j1 < H
        assert (j0 if v0 else 0) < H and (j1 if v1 else 0) < H
        i, part = (sc - mm * SP) >> 1, sc & 1
        if not v0 or i >= n_inst or mm >= mt:
            continue
        for j in [j0] + ([j1] if v1 else []):
            out += [(j, mm, i, part)] + ([(N - j, mm, i, part)] if j < half else [])
    return out, _issued(ntask, lambda t: (2 * H - 1) * (1 if t >= PT else 2))


def analysis_tasks(N, n_inst, mt, fp64):
    """Outputs written by one k_yanalysis CTA, [(even class, row, mode, instance, part)], and
    its issued FP64 multiply-adds (a pair: two chains of the class's length; a single row:
    one)."""
    H, half = N // 2 + 1, N // 2
    SP = col_pad(n_inst)
    SPt = SP * mt
    RW = 32 // SPt
    hE, hO = (H + 1) // 2, (half + 1) // 2
    loneE = fp64 and H % 2 == 1 and (hE - 1) % RW == 0
    loneO = fp64 and half % 2 == 1 and (hO - 1) % RW == 0
    assert not (loneE and loneO)
    pE, pO = hE - (1 if loneE else 0), hO - (1 if loneO else 0)
    ER, OR = round_up(pE, RW), round_up(pO, RW)
    PT = (ER + OR) * SPt
    ntask = PT + (SPt if (loneE or loneO) else 0)

    def kind(t):
        return ("single", loneE) if t >= PT else ("pair", (t // SPt) < ER)

    assert PT % 32 == 0 and _warps_uniform(ntask, kind)
    out = []
    for t in range(ntask):
        single = t >= PT
        sc = t - PT if single else t % SPt
        rs, mm = t // SPt, sc // SP
        even = loneE if single else rs < ER
        nrow, hh, pp = (H, hE, pE) if even else (half, hO, pO)
        k0 = hh - 1 if single else (rs if even else rs - ER)
        k1 = k0 + hh
        v0 = single or k0 < pp
        v1 = (not single) and v0 and k1 < nrow
        # rows of the staged tables (H x H each) and the state coefficient read
        assert (k0 if v0 else 0) < H and (k1 if v1 else 0) < H
        i, part = (sc - mm * SP) >> 1, sc & 1
        if i >= n_inst or mm >= mt:
            continue
        for ok, k in ((v0, k0), (v1, k1)):
            if ok:
                assert k < nrow and (2 * k if even else 2 * k + 1) <= N
                out.append((even, k, mm, i, part))

    def fma(t):
        single, even = kind(t)
        return (H if even else half) * (1 if single == "single" else 2)
    return out, _issued(ntask, fma)


GRIDS_N = list(range(8, 129, 2))   # ny = N + 1 odd, 9..129


def _tiles(n_inst):
    return [mt for mt in (1, 2, 4, 8, 16) if col_pad(n_inst) * mt <= 32]


@pytest.mark.parametrize("fp64", [True, False], ids=["fp64", "float_float"])
def test_synthesis_writes_every_value_once(fp64):
    for N, n_inst in itertools.product(GRIDS_N, range(1, 9)):
        for mt in _tiles(n_inst):
            got = synthesis_tasks(N, n_inst, mt, fp64)[0]
            want = {(y, mm, i, p) for y in range(N + 1) for mm in range(mt)
                    for i in range(n_inst) for p in range(2)}
            assert len(got) == len(set(got)) and set(got) == want, (N, n_inst, mt)


@pytest.mark.parametrize("fp64", [True, False], ids=["fp64", "float_float"])
def test_analysis_writes_every_coefficient_once(fp64):
    for N, n_inst in itertools.product(GRIDS_N, range(1, 9)):
        H, half = N // 2 + 1, N // 2
        for mt in _tiles(n_inst):
            got = analysis_tasks(N, n_inst, mt, fp64)[0]
            want = {(e, k, mm, i, p) for e in (True, False) for k in range(H if e else half)
                    for mm in range(mt) for i in range(n_inst) for p in range(2)}
            assert len(got) == len(set(got)) and set(got) == want, (N, n_inst, mt)


def test_unpaired_rows_cut_the_issued_work():
    """The FP64 map never issues more multiply-adds than the pair-only map (the float-float
    form), and issues fewer exactly when a class has an odd number of rows h and the middle
    row's pair would start a warp: the values and even coefficients for N = 0 mod 4
    (H = N/2 + 1 odd), the odd coefficients for N = 2 mod 4 (N/2 odd)."""
    for N in GRIDS_N:
        H, half = N // 2 + 1, N // 2
        for n_inst in range(1, 9):
            for mt in _tiles(n_inst):
                rw = 32 // (col_pad(n_inst) * mt)
                s64, sff = synthesis_tasks(N, n_inst, mt, True)[1], synthesis_tasks(N, n_inst, mt, False)[1]
                a64, aff = analysis_tasks(N, n_inst, mt, True)[1], analysis_tasks(N, n_inst, mt, False)[1]
                cut_s = H % 2 == 1 and ((H + 1) // 2 - 1) % rw == 0
                cut_a = cut_s or (half % 2 == 1 and ((half + 1) // 2 - 1) % rw == 0)
                assert (s64 < sff) if cut_s else (s64 == sff), (N, n_inst, mt)
                assert (a64 < aff) if cut_a else (a64 == aff), (N, n_inst, mt)
    # 32x33x32, groups of 4 instances (8 columns), 2 modes per CTA (16 columns, two rows of
    # pairs per warp).  Synthesis, H = 17 rows: pairs (j, j + 9) for j < 9, the last with a
    # dead partner: 10 pair rows x 16 columns = 5 warps of 2 (17 + 16) = 66 -> 330; with the
    # single row: 4 pair warps + 1 warp of 33 -> 297.  Analysis: 17 even rows (length 17) and
    # 16 odd rows (length 16): 5 even warps of 34 + 4 odd warps of 32 = 298 -> 4 x 34 + 4 x 32
    # + 1 x 17 = 281.
    assert synthesis_tasks(32, 4, 2, False)[1] == 330 and synthesis_tasks(32, 4, 2, True)[1] == 297
    assert analysis_tasks(32, 4, 2, False)[1] == 298 and analysis_tasks(32, 4, 2, True)[1] == 281
    # 32x31x32 (N = 30), same tiles: 15 odd-coefficient rows in 8 pairs, two pairs per warp;
    # the pair with the dead row (k = 7) shares its warp with k = 6, so no single-row tasks:
    # 16 even rows in 4 warps of 2 x 16 + 4 odd warps of 2 x 15 = 128 + 120 = 248
    assert analysis_tasks(30, 4, 2, True)[1] == analysis_tasks(30, 4, 2, False)[1] == 248
