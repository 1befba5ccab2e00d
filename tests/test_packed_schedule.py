"""The packed kernels' row schedules (ilu_packed_schedule), checked on the
CPU before any launch.

An emulator walks a schedule step by step with the packed kernel's data
flow -- a ring of the last 32 results per lane, a queue of 8 slots filled 7
steps ahead, results stored to the packed array at the end of each four-step
block, far producers read back from w in global memory, a lane switching rows
on the idle step before each row -- and with the oracle's FP64 surrogate
values computes one sweep x + C~^-1 (b - A x) (Alg. 2, V2).  Every value it
reads carries the point it belongs to and the step it was written at, so a
read of the wrong point, of a value not yet written, or of a ring slot
already overwritten fails.  The result must equal the oracle's sweep.
"""
import numpy as np
import pytest

import seeded_inputs as si

RING, SLOTS, PRE = 32, 8, 7


@pytest.fixture(scope="module")
def g():
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def decode(e):
    start, nyz, gb, rid, p0, p1, p2, _ = (int(v) for v in e)
    return start, (nyz >> 10) & 1023, nyz >> 20, [p0 & 0xffffffff, p1 & 0xffffffff, p2 & 0xffffffff]


def mode(c):
    return (c >> 30) & 3


def emulate_pass(N, T, lanes, rows, forward, Ls, Dinv, point_id, pw):
    """One substitution on the schedule with the packed kernel's data flow.
    pw: dict (forward step, lane) -> [value, point, pass, step] -- the packed
    array, holding the input of this pass at every point's slot.  The pass
    overwrites each point's slot with its result.  Returns nothing."""
    prow = (lambda s: s) if forward else (lambda s: T - 1 - s)
    tag = "f" if forward else "b"
    ring = {}                      # (step % RING, lane) -> (value, point, step)
    queue = {}                     # (step % SLOTS, lane) -> 4 x (value, point) or None
    state = [dict(prev=[None] * 3, v1=None) for _ in range(lanes)]
    ptr = {}

    def point_at(lane, tau, which):
        """(row entry, u) the lane works on at step tau, u = 0 the idle step
        (steps are asked for in increasing order per lane and `which`)."""
        k = ptr.get((lane, which), 0)
        rl = rows[lane]
        while k < len(rl) and tau > rl[k][0] + (N - 1 - rl[k][1] - rl[k][2]) - 1:
            k += 1
        ptr[(lane, which)] = k
        if k < len(rl) and rl[k][0] - 1 <= tau:
            return rl[k], tau - rl[k][0] + 1
        return None, None

    def neighbours(y, z, x, j):
        """grid coordinates of the first and second value of producer j"""
        if forward:
            return [((x, y - 1, z), (x + 1, y - 1, z)), ((x, y, z - 1), (x + 1, y, z - 1)),
                    ((x - 1, y + 1, z - 1), (x, y + 1, z - 1))][j]
        return [((x, y + 1, z), (x - 1, y + 1, z)), ((x, y, z + 1), (x - 1, y, z + 1)),
                ((x + 1, y - 1, z + 1), (x, y - 1, z + 1))][j]

    def interior(p):
        return p[0] >= 1 and p[1] >= 1 and p[2] >= 1 and sum(p) <= N - 1

    for tau in range(-PRE, T):
        # phase 1: every lane prefetches for step tau + PRE (before any write of step tau)
        for lane in range(lanes):
            t2 = tau + PRE
            r, u = point_at(lane, t2, 0)
            if r is None:
                continue
            start, y, z, codes = r
            n = N - 1 - y - z
            x = u if forward else n + 1 - u
            ent_q = [None] * 4
            if u >= 1:
                e = pw[(prow(t2), lane)]
                assert e[1] == (x, y, z) and e[2] != tag, "input slot holds another point or was overwritten"
                ent_q[0] = (e[0], e[1])
            for j in range(3):
                if mode(codes[j]) != 2:
                    continue
                slot, k0 = codes[j] & 511, (codes[j] >> 9) & 0x1fffff
                e = pw.get((prow(t2 - k0 + 1), slot))  # a slot without a point: garbage, must be masked
                if e is not None and e[2] == tag:
                    # results reach global memory at the end of their four-step block
                    assert (e[3] | 3) + 1 <= tau, "far value read before it was stored"
                    ent_q[1 + j] = (e[0], e[1])
            queue[(t2 % SLOTS, lane)] = ent_q
        if tau < 0:
            continue
        # phase 2: every lane computes its point of step tau
        writes = []
        for lane in range(lanes):
            r, u = point_at(lane, tau, 1)
            st = state[lane]
            if r is None:
                continue
            start, y, z, codes = r
            n = N - 1 - y - z
            qv = queue[(tau % SLOTS, lane)]
            # each producer's second value of this step; the first is the one
            # carried from the step before, as in the kernel
            second = []
            for j in range(3):
                md = mode(codes[j])
                if md == 1:
                    slot, k0 = codes[j] & 511, (codes[j] >> 9) & 31
                    e = ring.get(((tau - k0 + 1) % RING, slot))
                    second.append(e if e is not None and e[2] == tau - k0 + 1 else None)
                elif md == 2:
                    second.append(qv[1 + j])
                else:
                    second.append(None)
            carried = st["prev"]
            st["prev"] = second
            if u == 0:
                continue
            x = u if forward else n + 1 - u
            p = (x, y, z)
            vals = []
            for j in range(3):
                a, bb = neighbours(y, z, x, j)
                f, sv = carried[j], second[j]
                vals.append((a, f[0] if f and f[1] == a else None, bb, sv[0] if sv and sv[1] == bb else None))

            def use(point, value):
                if not interior(point):
                    return 0.0
                assert value is not None, f"step {tau}: value of {point} missing or wrong for {p}"
                return value

            if forward:
                acc = qv[0][0]
                Lp = lambda d: Ls[d][point_id(*p)]
                terms = [(1, use(vals[0][0], vals[0][1])), (2, use(vals[0][2], vals[0][3])),
                         (3, use(vals[2][0], vals[2][1])), (4, use(vals[2][2], vals[2][3])),
                         (5, use(vals[1][0], vals[1][1])), (6, use(vals[1][2], vals[1][3]))]
                for d, v in terms:  # d: w s se bnw bn bc be = 0..6 (the paper's D_l)
                    acc -= Lp(d) * v
                own = (x - 1, y, z)
                if interior(own):
                    acc -= Lp(0) * st["v1"]
            else:
                acc = Dinv[point_id(*p)] * qv[0][0]

                def Lq(d, q):  # L~^{p-d}_d at q = p - d
                    return Ls[d][point_id(*q)] if interior(q) else 0.0
                acc -= Lq(1, vals[0][0]) * use(vals[0][0], vals[0][1])   # p - s
                acc -= Lq(5, vals[1][0]) * use(vals[1][0], vals[1][1])   # p - bc
                acc -= Lq(3, vals[2][0]) * use(vals[2][0], vals[2][1])   # p - bnw
                acc -= Lq(2, vals[0][2]) * use(vals[0][2], vals[0][3])   # p - se
                acc -= Lq(6, vals[1][2]) * use(vals[1][2], vals[1][3])   # p - be
                acc -= Lq(4, vals[2][2]) * use(vals[2][2], vals[2][3])   # p - bn
                own = (x + 1, y, z)
                if interior(own):
                    acc -= Lq(0, own) * st["v1"]
            writes.append((lane, acc, p))
            st["v1"] = acc
        for lane, acc, p in writes:
            ring[(tau % RING, lane)] = (acc, p, tau)
            key = (prow(tau), lane)
            assert pw[key][1] == p, "result written to another point's slot"
            pw[key] = [acc, p, tag, tau]


@pytest.mark.parametrize("level,lanes", [(3, 0), (4, 0), (5, 0), (5, 24), (6, 48), (6, 0)])
def test_emulated_schedule_sweep_equals_the_oracle(g, orc, level, lanes):
    """Level 3-6 on the kernels' 384 lanes and on few lanes (which forces
    long delays and far producers read from global memory): the emulated
    sweep equals the oracle's sweep to FP64 rounding."""
    P = si.macro_tet(60 + level)
    co = orc.Coeff("sinprod", 1.0, 0.5)
    pr = orc.Problem(P, level, co, deg=[3, 3, 3])
    N = pr.N
    Ls, Dinv = pr.surrogate_factors()
    ids, _ = orc.interior_ids(N)
    point_id = lambda x, y, z: ids[orc.index(N, x, y, z)]
    x0 = si.boundary_data(level, 61)
    b = si.rhs(level, 62)
    want = orc.smooth(pr.A, N, Ls, Dinv, x0.copy(), b, 1)
    r, _ = orc.residual(pr.A, N, x0, b)
    T, ln, ent_f, off = g.packed_schedule(level, True, lanes)
    _, _, ent_b, off_b = g.packed_schedule(level, False, lanes)
    assert np.array_equal(off, off_b)
    rows_f = [[decode(ent_f[e]) for e in range(off[l], off[l + 1])] for l in range(ln)]
    rows_b = [[decode(ent_b[e]) for e in range(off[l], off[l + 1])] for l in range(ln)]
    # the packed array: r of every point at (forward step of the point, lane)
    pw = {}
    for l in range(ln):
        for start, y, z, _ in rows_f[l]:
            for x in range(1, N - y - z):
                pw[(start + x - 1, l)] = [r[orc.index(N, x, y, z)], (x, y, z), "r", -1]
    emulate_pass(N, T, ln, rows_f, True, Ls, Dinv, point_id, pw)
    emulate_pass(N, T, ln, rows_b, False, Ls, Dinv, point_id, pw)
    x = x0.copy()
    for (s_, l), (v, p, tag, _) in pw.items():
        assert tag == "b"
        x[orc.index(N, *p)] += v
    assert np.abs(x - want).max() <= 1e-12 * np.abs(want).max()
    far = sum(int(mode(int(c) & 0xffffffff) == 2) for e in np.concatenate([ent_f, ent_b]) for c in e[4:7])
    if lanes and level >= 6:
        assert far > 0  # the run exercised the global-memory path


@pytest.mark.parametrize("level", [5, 7, 8])
def test_schedule_covers_every_row_once(g, orc, level):
    """Each interior row appears once per pass on the same lane; a lane's rows
    follow one another with the idle step and the coefficient-copy distance
    the kernel relies on, in both passes; the backward pass is the forward
    one reversed in time."""
    N = 2 ** level
    T, ln, ef, off = g.packed_schedule(level, True)
    _, _, eb, _ = g.packed_schedule(level, False)
    for ent in (ef, eb):
        rows = {((int(e[1]) >> 10) & 1023, int(e[1]) >> 20) for e in ent}
        assert len(rows) == len(ent) == (N - 3) * (N - 2) // 2
        for l in range(ln):
            prev_start = prev_n = None
            for e in ent[off[l]:off[l + 1]]:
                start, y, z = int(e[0]), (int(e[1]) >> 10) & 1023, int(e[1]) >> 20
                n = N - 1 - y - z
                assert int(e[1]) & 1023 == n and int(e[2]) == orc.index(N, 0, y, z)
                assert start >= 1 and start + n <= T
                if prev_start is not None:
                    assert start >= prev_start + max(prev_n + 1, PRE + 2)
                prev_start, prev_n = start, n
    for l in range(ln):
        fw = [(int(e[0]), int(e[1])) for e in ef[off[l]:off[l + 1]]]
        bw = [(int(e[0]), int(e[1])) for e in eb[off[l]:off[l + 1]]]
        assert [yz for _, yz in bw] == [yz for _, yz in reversed(fw)]
        assert [s for s, _ in bw] == [T - s - (yz & 1023) for s, yz in reversed(fw)]
