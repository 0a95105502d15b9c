"""Host replay of the index maps of two Stokes-solve organisations (§4 steps 1 and 4).

- The banded sweeps with one thread per chain (k_sweep): thread q of an instance's launch runs
  chain (group g, mode m, part rho) = (q >> 1 divided by the run's mode count, its remainder,
  q & 1).  For every grid the library accepts, both launch widths and the full and reduced
  (modes m >= 0) launches: every chain of the run exists exactly once, the two parts of a mode
  sit on neighbouring lanes of one warp, every output coefficient (component, mode, n, part) is
  written exactly once, and every class array index stays inside its Mh slots.
- The dense per-mode solve of the per-mode kernel: task t of a CTA holding nmod modes is a
  v row (list A) or a pair of eta rows (list B), both run as two operator segments.  For every
  accepted ny and tile: every v row, eta row and mean-mode u / w row of every mode is written
  exactly once, each row's chain covers its class length, and the operator rows read are
  inside their Mh x Mh blocks.
They need no GPU and do not use the oracle."""
import pytest

GRID_NY = list(range(9, 130, 2))  # every accepted ny (odd, 9..129)


def _mh(ny):
    return (ny - 1) // 2 + 1


def _class_len(N, par):
    return (N - par) // 2 + 1


def _sweep_ctas(nrun, threads):
    return (4 * nrun + threads - 1) // threads


def _sweep_outputs(N, g, m, rho, mean):
    """Outputs (component, mode, n, part) of one chain, as the kernel assembles them."""
    out = []
    if mean:
        Mc = _class_len(N, g)
        for i in range(Mc):
            for comp in range(3):
                out.append((comp, m, g + 2 * i, rho))
        return out
    pv, pP = g, 1 - g
    out += [(1, m, pv + 2 * i, rho) for i in range(_class_len(N, pv))]
    for i in range(_class_len(N, pP)):
        out.append((0, m, pP + 2 * i, rho))
        out.append((2, m, pP + 2 * i, rho))
    return out


@pytest.mark.parametrize("threads", [32, 64])
@pytest.mark.parametrize("reduced", [False, True])
@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32), (32, 31, 32), (48, 49, 48), (32, 17, 48),
                                  (64, 65, 64), (128, 97, 128), (24, 129, 24)])
def test_sweep_chain_map(grid, threads, reduced):
    nx, ny, nz = grid
    N, Mh = ny - 1, _mh(ny)
    Kx, Kz = nx // 3 - 1, nz // 3 - 1
    Mx, Mz = 2 * Kx + 1, Kz + 1
    nm = Mx * Mz
    nr = (Kx + 1) * Mz if reduced else nm
    ctas = _sweep_ctas(nr, threads)
    chains, outputs = set(), {}
    for cta in range(ctas):
        for lane in range(threads):
            q = cta * threads + lane
            if q >= 4 * nr:
                continue
            rho, gm = q & 1, q >> 1
            g, m = gm // nr, gm % nr
            assert g in (0, 1) and 0 <= m < nr
            # the partner part: the neighbouring lane of the same warp, same (g, m)
            qp = q ^ 1
            assert qp // 32 == q // 32 and qp // threads == q // threads
            assert (qp >> 1) == gm
            assert (g, m, rho) not in chains
            chains.add((g, m, rho))
            for i in range(Mh):  # every class array of the chain fits its Mh slots
                assert i * threads + lane < Mh * threads
            for o in _sweep_outputs(N, g, m, rho, m == 0):
                outputs[o] = outputs.get(o, 0) + 1
    assert len(chains) == 4 * nr
    # every coefficient n = 0..N of the three components of every run mode, both parts, once
    assert len(outputs) == 3 * nr * ny * 2
    assert all(v == 1 for v in outputs.values())
    assert all(0 <= o[2] <= N for o in outputs)


@pytest.mark.parametrize("ny", GRID_NY)
@pytest.mark.parametrize("nmod", [1, 2, 3, 4, 6])
def test_dense_two_segment_task_map(ny, nmod):
    N, Mh = ny - 1, _mh(ny)
    HB = (Mh + 1) // 2
    nA, nB = nmod * 2 * Mh, nmod * 2 * HB
    for mean_mode in (False, True):
        writes = {}
        for t in range(nA + nB):
            isA = t < nA
            tt = t if isA else t - nA
            per = Mh if isA else HB
            r, q = tt % per, tt // per
            g, mm = q & 1, q >> 1
            assert 0 <= mm < nmod
            pv, pP = g, 1 - g
            McV, McP = _class_len(N, pv), _class_len(N, pP)
            mean = mean_mode and mm == 0
            segs = []  # (operator block, row, length, output or None)
            if mean:
                Mc = _class_len(N, g)
                if r < Mc:
                    segs.append(("Eh", r, Mc, ("u" if isA else "w", mm, g, r)))
                if not isA and r + HB < Mc:
                    segs.append(("Eh", r + HB, Mc, ("w", mm, g, r + HB)))
            elif isA:
                if r < McV:
                    segs.append(("Av", r, McV, None))
                    segs.append(("Ag", r, McP, ("v", mm, g, r)))
            else:
                if r < McP:
                    segs.append(("Eh", r, McP, ("eta", mm, g, r)))
                if r + HB < McP:
                    segs.append(("Eh", r + HB, McP, ("eta", mm, g, r + HB)))
            for blk, row, n, out in segs:
                assert 0 <= row < Mh and 0 < n <= Mh
                if out is not None:
                    writes[out] = writes.get(out, 0) + 1
        want = set()
        for mm in range(nmod):
            for g in (0, 1):
                if mean_mode and mm == 0:
                    Mc = _class_len(N, g)
                    want |= {("u", mm, g, r) for r in range(Mc)} | {("w", mm, g, r) for r in range(Mc)}
                else:
                    want |= {("v", mm, g, r) for r in range(_class_len(N, g))}
                    want |= {("eta", mm, g, r) for r in range(_class_len(N, 1 - g))}
        assert set(writes) == want
        assert all(v == 1 for v in writes.values())
