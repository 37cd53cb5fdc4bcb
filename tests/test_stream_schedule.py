"""The schedules of the streaming band kernels (stream2d.cu, stream9.cu), emulated on
the CPU (no arithmetic).

Each emulation replays a run of a CTA (the strips [ya, yb) of one band) step by
step with the kernels' row windows, column windows, barrier intervals, TMA block
issue points and ring sizes, and tracks for every site which colour phase last
wrote it and whether every value it read was the one a global colour sweep gives.
It checks that:
  - every stored final row of the run is correct (the first step's recomputed rows
    and the band halo never leak into it);
  - every coarse site of the run is restricted from correct residual rows, and the
    residual ring still holds those rows when the restriction reads them;
  - a ring slot is only overwritten by a new TMA block after the barrier that ends
    the last interval reading it, and every row read lies in the block its slot holds.
The 5-point kernels are red-black (forward: red, black, residual; the backward's red
phase runs beside the next step's prolongation); the 9-point kernels use the four
parity colours (0,0), (1,1), (0,1), (1,0) forward and the reverse backward (P3 of
the backward beside the next prolongation).  Planted schedule errors (a column
window one column short, a 32-row residual ring) fail these checks.
"""
import pytest

K = 16   # rows per step (strip)
BK = 8   # rows per TMA block


def cdiv_pos(a, b):
    return (a + b - 1) // b if a > 0 else 0


class Ring:
    """TMA ring of nb slots of BK-row blocks starting at row `base`."""

    def __init__(self, base, nb, first_issue):
        self.base, self.nb = base, nb
        self.slot = {k % nb: k for k in range(first_issue + 1)}

    def check(self, j, lo=None, hi=None):
        if j - self.base < 0:
            return None          # rows above the run: stale ring rows, read only by recomputed rows
        k = (j - self.base) // BK
        assert self.slot.get(k % self.nb) == k, ("ring slot holds another block", j, k)
        if lo is not None:
            assert lo <= k <= hi, ("row outside the step's blocks", j, k, lo, hi)
        return k

    def issue(self, k):
        self.slot[k % self.nb] = k


# ----------------------------------------------------------------------------
# 5-point kernels (stream2d.cu): 128-column bands, 8-slot ring, 64-row residual ring
# ----------------------------------------------------------------------------
BW5, NB5, RR5 = 128, 8, 64


def _red(i, j):
    return (i + j) % 2 == 0


def emulate5_fwd(n, ya, yb, x0, rring=RR5, red_lo=2):
    nc = (n - 1) // 2
    ver, ok = {}, {}

    def get(i, j):
        if not (0 <= i < n and 0 <= j < n):
            return None
        return ver.get((i, j), 0), ok.get((i, j), True)

    def update(i, j, black):
        good = True
        for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            ring.check(j + dj)
            t = get(i + di, j + dj)
            if t is not None and (t[0] != (1 if black else 0) or not t[1]):
                good = False        # red reads old black, black reads new red
        assert ver.get((i, j), 0) == 0
        ver[(i, j)], ok[(i, j)] = 1, good

    def final(i, j):
        t = get(i, j)
        return t is None or (t[0] == 1 and t[1])

    jend = yb >> 1
    S = max(max(cdiv_pos(yb - ya - (K - 2), K), cdiv_pos(jend - (ya >> 1) - (K // 2 - 3), K // 2)) + 1, 1)
    KB = 2 * S
    ring = Ring(ya - 3, NB5, min(KB, 4))
    resid, rslot, stored, restricted = {}, {}, {}, set()

    def residual(t):
        R = ya - 2 + K * t
        for rp in range(K // 2):
            for j in (R + 2 * rp - 2, R + 2 * rp - 1):
                for dj in (-1, 0, 1):
                    ring.check(j + dj)
                for i in range(x0, x0 + BW5 + 4):
                    if 0 <= j < n and i < n:
                        resid[(i, j)] = all(final(i + di, j + dj) for di, dj in
                                            ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)))
                    else:
                        resid[(i, j)] = True
                rslot[(j - ya + 4) % rring] = j

    def restrict(t):
        for cj in range(8):
            Jc = ((ya - 2 + K * t) >> 1) - 2 + cj
            for ci in range(32):
                I = (x0 >> 1) + 2 * ci
                if not I < nc or Jc < (ya >> 1) or Jc >= jend:
                    continue
                for b in range(3):
                    rr = 2 * Jc + b
                    assert rslot.get((rr - ya + 4) % rring) == rr, ("residual ring row reused", rr)
                    assert all(resid.get((c, rr)) for c in range(2 * I, 2 * I + 5)), ("residual", I, rr)
                restricted.update({(I, Jc), (I + 1, Jc)} if I + 1 < nc else {(I, Jc)})

    for s in range(S):
        R = ya - 2 + K * s
        for k in range(2 * s + 5, min(2 * s + 6, KB) + 1):
            ring.issue(k)          # at the top of the step, after the barrier
        for rp in range(K // 2):   # red on rows ja, ja + 1
            for j in (R + 2 * rp, R + 2 * rp + 1):
                if 0 <= j < n:
                    for i in range(max(x0 - red_lo, 0), min(x0 + BW5 + 3, n)):
                        if _red(i, j):
                            update(i, j, False)
        for rp in range(K // 2):   # black on rows ja - 1, ja; stores
            for j in (R + 2 * rp - 1, R + 2 * rp):
                if 0 <= j < n:
                    for i in range(max(x0 - 1, 0), min(x0 + BW5 + 2, n)):
                        if not _red(i, j):
                            update(i, j, True)
                if ya <= j < yb:
                    for i in range(x0, min(x0 + BW5, n)):
                        stored[(i, j)] = final(i, j)
        residual(s)                # the restriction of the previous step reads in the same interval
        if s > 0:
            restrict(s - 1)
    restrict(S - 1)
    assert all(stored.get((i, j)) for j in range(ya, yb) for i in range(x0, min(x0 + BW5, n)))
    assert all((I, J) in restricted for J in range(ya >> 1, min(jend, nc))
               for I in range(x0 >> 1, min((x0 >> 1) + BW5 // 2, nc)))


def emulate5_bwd(n, ya, yb, x0):
    ver, ok, prol = {}, {}, set()

    def get(i, j):
        if not (0 <= i < n and 0 <= j < n):
            return None
        return ver.get((i, j), 0), ok.get((i, j), True) and (i, j) in prol

    def update(i, j, black):
        good = (i, j) in prol
        for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            ring.check(j + dj)
            t = get(i + di, j + dj)
            if t is not None and (t[0] != (0 if black else 1) or not t[1]):
                good = False        # backward: black first (old red), red reads new black
        assert ver.get((i, j), 0) == 0
        ver[(i, j)], ok[(i, j)] = 1, good

    def final(i, j):
        t = get(i, j)
        return t is None or (t[0] == 1 and t[1])

    S = cdiv_pos(yb - ya - (K - 4), K) + 1
    KB = 2 * S
    ring = Ring(ya - 2, NB5, min(KB, 4))
    stored = {}

    def red(t):
        R = ya - 2 + K * t
        for rp in range(K // 2):
            for j in (R + 2 * rp - 2, R + 2 * rp - 1):
                if 0 <= j < n:
                    for i in range(max(x0, 0), min(x0 + BW5, n)):
                        if _red(i, j):
                            update(i, j, False)
                if ya <= j < yb:
                    for i in range(x0, min(x0 + BW5, n)):
                        stored[(i, j)] = final(i, j)

    for s in range(S):
        R = ya - 2 + K * s
        for rp in range(K // 2):   # prolongation on rows ja, ja + 1 (all staged groups)
            for j in (R + 2 * rp, R + 2 * rp + 1):
                if 0 <= j < n:
                    ring.check(j)
                    for i in range(max(x0 - 4, 0), min(x0 + BW5 + 4, n)):
                        assert (i, j) not in prol
                        prol.add((i, j))
        if s > 0:
            red(s - 1)             # beside the prolongation
        for k in range(2 * s + 5, min(2 * s + 6, KB) + 1):
            ring.issue(k)          # after the barrier that ends the first interval
        for rp in range(K // 2):   # black on rows ja - 1, ja
            for j in (R + 2 * rp - 1, R + 2 * rp):
                if 0 <= j < n:
                    for i in range(max(x0 - 1, 0), min(x0 + BW5 + 1, n)):
                        if not _red(i, j):
                            update(i, j, True)
    red(S - 1)
    assert all(stored.get((i, j)) for j in range(ya, yb) for i in range(x0, min(x0 + BW5, n)))


def _runs(n, bw, full=False):
    spb = (n + K - 1) // K
    for band in range((n + bw - 1) // bw):
        pairs = [(0, spb), (0, 1), (1, 3), (spb - 1, spb), (2, spb)]
        if full:
            pairs = [(a, b) for a in range(spb) for b in range(a + 1, spb + 1)]
        for s0, s1 in pairs:
            if 0 <= s0 < s1 <= spb:
                yield K * s0, min(K * s1, n), bw * band


@pytest.mark.parametrize("n", [63, 127, 255])
def test_five_point_schedule(n):
    for ya, yb, x0 in _runs(n, BW5, full=n == 63):
        emulate5_fwd(n, ya, yb, x0)
        emulate5_bwd(n, ya, yb, x0)


def test_five_point_schedule_catches_planted_errors():
    with pytest.raises(AssertionError):   # red window one column short on the left
        emulate5_fwd(255, 0, 64, 128, red_lo=1)


# ----------------------------------------------------------------------------
# 9-point kernels (stream9.cu): 64-column bands, 5-slot ring, 64-row residual ring
# ----------------------------------------------------------------------------
BW9, NB9, RR9 = 64, 5, 64
FWD_ORDER = (0, 3, 2, 1)   # colour c = (i & 1) | (j & 1) << 1
BWD_ORDER = (1, 2, 3, 0)


def _colour(i, j):
    return (i & 1) | ((j & 1) << 1)


def _emulate9(n, ya, yb, x0, fwd, rring=RR9, lag0=4):
    nc = (n - 1) // 2
    order = FWD_ORDER if fwd else BWD_ORDER
    phase_of = {c: p for p, c in enumerate(order)}
    ver, ok, prol = {}, {}, set()
    jend = yb >> 1
    if fwd:
        S = max(max(cdiv_pos(yb - ya - (K - 4), K), cdiv_pos(jend - (ya >> 1) - (K // 2 - 3), K // 2)) + 1, 1)
        R0, base = ya - 2, ya - 6
        # P0 .. P3 column windows, widening by one column per earlier phase (residual [x0, x0 + 64])
        wins = [(x0 - lag0 + p, x0 + BW9 + 4 - p) for p in range(4)]
    else:
        S = cdiv_pos(yb - ya - (K - 6), K) + 1
        R0, base = ya - 4, ya - 7
        wins = [(x0 - 3 + p, x0 + BW9 + 2 - p) for p in range(4)]
    KB = 2 * S
    ring = Ring(base, NB9, min(KB, NB9 - 1))

    def get(i, j):
        if not (0 <= i < n and 0 <= j < n):
            return None
        return ver.get((i, j), 0), ok.get((i, j), True) and (fwd or (i, j) in prol)

    def final(i, j):
        t = get(i, j)
        return t is None or (t[0] == 1 and t[1])

    def phase(p, t):
        """colour phase p of step t on its rows: P0 row a, P1/P2 row a - 1, P3 row a - 2"""
        R = R0 + K * t
        lo, hi = wins[p]
        for rp in range(K // 2):
            a = R + 2 * rp
            j = (a, a - 1, a - 1, a - 2)[p]
            if not 0 <= j < n:
                continue
            for i in range(max(lo, 0), min(hi, n - 1) + 1):
                if _colour(i, j) != order[p]:
                    continue
                good = fwd or (i, j) in prol
                for dj in (-1, 0, 1):
                    ring.check(j + dj, 2 * t, min(2 * t + 2, KB))
                    for di in (-1, 0, 1):
                        if di or dj:
                            v = get(i + di, j + dj)
                            want = 1 if phase_of[_colour(i + di, j + dj)] < p else 0
                            if v is not None and (v[0] != want or not v[1]):
                                good = False
                assert ver.get((i, j), 0) == 0
                ver[(i, j)], ok[(i, j)] = 1, good
            if p in (2, 3) and ya <= (a - 1 if p == 2 else a - 2) < yb:
                jj = a - 1 if p == 2 else a - 2
                for i in range(x0, min(x0 + BW9, n)):
                    stored[(i, jj)] = final(i, jj)

    stored, resid, rslot, restricted = {}, {}, {}, set()

    def residual(t):
        R = R0 + K * t
        for rp in range(K // 2):
            for j in (R + 2 * rp - 3, R + 2 * rp - 2):
                for dj in (-1, 0, 1):
                    ring.check(j + dj, 2 * t, min(2 * t + 2, KB))
                for i in range(x0, x0 + BW9 + 8):
                    resid[(i, j)] = (not (0 <= j < n and i < n)) or all(
                        final(i + di, j + dj) for di in (-1, 0, 1) for dj in (-1, 0, 1))
                rslot[(j - ya + 8) % rring] = j

    def restrict(t):
        for cj in range(8):
            Jc = (ya >> 1) - 3 + (K // 2) * t + cj
            for ci in range(16):
                I = (x0 >> 1) + 2 * ci
                if not I < nc or Jc < (ya >> 1) or Jc >= jend:
                    continue
                for b in range(3):
                    rr = 2 * Jc + b
                    assert rslot.get((rr - ya + 8) % rring) == rr, ("residual ring row reused", rr)
                    assert all(resid.get((c, rr)) for c in range(2 * I, 2 * I + 5)), ("residual", I, rr)
                restricted.update({(I, Jc), (I + 1, Jc)} if I + 1 < nc else {(I, Jc)})

    for s in range(S):
        R = R0 + K * s
        if fwd:
            if s > 0:               # at the top of the step, after the barrier
                for k in range(2 * s + 3, min(2 * s + 4, KB) + 1):
                    ring.issue(k)
            for p in range(4):
                phase(p, s)
            residual(s)             # the restriction of the previous step reads in the same interval
            if s > 0:
                restrict(s - 1)
        else:
            for rp in range(K // 2):   # prolongation on rows a, a + 1 (staged groups inside the grid)
                for j in (R + 2 * rp, R + 2 * rp + 1):
                    if 0 <= j < n:
                        ring.check(j, 2 * s, min(2 * s + 2, KB))
                        for i in range(max(x0 - 4, 0), min(x0 + BW9 + 8, n)):
                            assert (i, j) not in prol
                            prol.add((i, j))
            if s > 0:
                phase(3, s - 1)         # P3 of the previous step beside the prolongation
                for k in range(2 * s + 3, min(2 * s + 4, KB) + 1):
                    ring.issue(k)       # after the barrier that ends the first interval
            for p in range(3):
                phase(p, s)
    if fwd:
        restrict(S - 1)
        assert all((I, J) in restricted for J in range(ya >> 1, min(jend, nc))
                   for I in range(x0 >> 1, min((x0 >> 1) + BW9 // 2, nc)))
    else:
        phase(3, S - 1)
    assert all(stored.get((i, j)) for j in range(ya, yb) for i in range(x0, min(x0 + BW9, n)))


@pytest.mark.parametrize("n", [63, 127, 255])
def test_nine_point_schedule(n):
    for ya, yb, x0 in _runs(n, BW9, full=n == 63):
        _emulate9(n, ya, yb, x0, fwd=True)
        _emulate9(n, ya, yb, x0, fwd=False)


def test_nine_point_schedule_catches_planted_errors():
    with pytest.raises(AssertionError):   # a 32-row residual ring
        _emulate9(127, 0, 127, 0, fwd=True, rring=32)
    with pytest.raises(AssertionError):   # P0 window one column short
        _emulate9(127, 0, 64, 64, fwd=True, lag0=3)
