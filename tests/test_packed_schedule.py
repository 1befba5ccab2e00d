"""The packed kernels' row schedules (ilu_packed_schedule), checked on the
CPU before any launch.

An emulator walks a schedule step by step with the packed kernel's data
flow -- a ring of the last 32 results per lane, a queue of 8 slots filled 7
steps ahead, results stored to the packed array at the end of each four-step
block, far producers read back from w in global memory, a lane switching rows
on the step before each row, every step without a point writing 0, the lanes
meeting at a barrier only every B steps -- and with the oracle's FP64
surrogate values computes one sweep x + C~^-1 (b - A x) (Alg. 2, V2).  Like
the kernel it reads every producer value without masks: each value carries
the point it belongs to and the step it was written at, so a read of the
wrong point, of a value not yet visible, or of a ring slot already
overwritten fails, and so does a read of a missing neighbour (outside the
interior) that does not give 0.  The result must equal the oracle's sweep.
"""
import numpy as np
import pytest

import seeded_inputs as si

RING, SLOTS, PRE, LANES, CLUSTER_LANES, BLOCK = 32, 8, 7, 384, 2 * 320, 8


@pytest.fixture(scope="module")
def g():
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def decode(e):
    """(switch step, first point step, n, y, z, producer codes, ring words,
    far bits, row id, t at the switch step) of a schedule entry"""
    w = [int(v) & 0xffffffff for v in e]
    sw, lo = w[0] & 0xffff, (w[0] & 0xffff) + ((w[0] >> 16) & 15)
    gm = (w[0] >> 20) & 7
    n, y, z = w[1] & 1023, (w[1] >> 10) & 1023, w[1] >> 20
    R = [w[2] & 0x7fff, (w[2] >> 15) & 0x7fff, w[3] & 0x7fff]
    rid = (w[3] >> 15) & 0x7fff
    tt0 = float(np.array([w[4]], dtype=np.uint32).view(np.float32)[0])
    return dict(sw=sw, lo=lo, n=n, y=y, z=z, codes=w[5:8], R=R, gm=gm, rid=rid, tt0=tt0)


def lane_k0(c):
    """the producer's lane and the step distance k0 of a producer code"""
    return c & 1023, (c >> 10) & 0xfffff


def mode(c):
    return (c >> 30) & 3


def quantum_of(level):
    return 1 if level <= 6 else (2 if level == 7 else 4)


def lanes_of(level):
    return LANES if level <= 7 else CLUSTER_LANES


def emulate_pass(N, T, lanes, rows, forward, Ls, Dinv, point_id, pw, B=1):
    """One substitution on the schedule with the packed kernel's data flow,
    the CTA meeting at a barrier after every step B - 1 (mod B): a ring value
    read at step tau must have been written before the barrier that opened
    tau's group of B steps, and its ring row must not be rewritten by any
    step of that group (lanes may be up to B - 1 steps apart).
    pw: dict (forward step, lane) -> [value, point or None, pass, step] --
    the packed array with every slot (a slot without a point holds 0); the
    pass overwrites every slot with its result (0 without a point)."""
    prow = (lambda s: s) if forward else (lambda s: T - 1 - s)
    tag = "f" if forward else "b"
    ring = {}                      # (step % RING, lane) -> (value, point or None, step)
    queue = {}                     # (step % SLOTS, lane) -> 3 x (value, point or None) or None
    state = [dict(prev=[(0.0, None)] * 3, v1=0.0, v1p=None) for _ in range(lanes)]
    ptr = {}
    pending = []                   # block stores not yet issued: (step, lane, value, point)

    def point_at(lane, tau, which):
        """the row entry the lane holds at step tau: from its switch step to
        its last point (steps are asked for in increasing order per lane and
        `which`)"""
        k = ptr.get((lane, which), 0)
        rl = rows[lane]
        while k < len(rl) and tau > rl[k]["lo"] + rl[k]["n"] - 1:
            k += 1
        ptr[(lane, which)] = k
        if k < len(rl) and rl[k]["sw"] <= tau:
            return rl[k]
        return None

    def neighbours(y, z, x, j):
        """grid coordinates of the first and second value of producer j"""
        if forward:
            return [((x, y - 1, z), (x + 1, y - 1, z)), ((x, y, z - 1), (x + 1, y, z - 1)),
                    ((x - 1, y + 1, z - 1), (x, y + 1, z - 1))][j]
        return [((x, y + 1, z), (x - 1, y + 1, z)), ((x, y, z + 1), (x - 1, y, z + 1)),
                ((x + 1, y - 1, z + 1), (x, y - 1, z + 1))][j]

    def interior(p):
        return p[0] >= 1 and p[1] >= 1 and p[2] >= 1 and sum(p) <= N - 1

    def checked(want, got):
        """the value the kernel uses for neighbour `want` (no mask)"""
        value, point = got
        if interior(want):
            assert point == want, f"read {point} for {want}"
        else:
            assert value == 0.0, f"missing neighbour {want} read as {value} ({point})"
        return value

    for tau in range(-PRE, T):
        # phase 1: every lane prefetches its far values for step tau + PRE
        for lane in range(lanes):
            t2 = tau + PRE
            r = point_at(lane, t2, 0)
            if r is None:
                continue
            codes = r["codes"]
            ent_q = [None] * 3
            for j in range(3):
                if mode(codes[j]) != 2:
                    continue
                slot, k0 = lane_k0(codes[j])
                e = pw[(prow(t2 - k0 + 1), slot)]
                if e[2] == tag:  # written in this pass: stored at the end of its four-step block
                    assert (e[3] | 3) + 1 <= tau, "far value read before it was stored"
                ent_q[j] = (e[0], e[1])
            queue[(t2 % SLOTS, lane)] = ent_q
        if tau < 0:
            continue
        # phase 2: every lane computes its point of step tau, or 0
        writes = []
        for lane in range(lanes):
            r = point_at(lane, tau, 1)
            st = state[lane]
            if r is None:  # no row now: the lane's registers are stale, its result 0
                writes.append((lane, 0.0, None))
                continue
            y, z, codes, n = r["y"], r["z"], r["codes"], r["n"]
            u = tau - r["lo"] + 1  # the point's index in the pass (<= 0: the switch or an idle step)
            qv = queue.get((tau % SLOTS, lane))
            second = []  # each producer's second value of this step; the first is carried
            for j in range(3):
                md = mode(codes[j])
                if md == 1:
                    slot, k0 = lane_k0(codes[j])
                    w, g0 = tau - k0 + 1, tau - tau % B
                    assert w < g0, "ring value read in the group of steps that wrote it"
                    assert w + RING > g0 + B - 1, "ring row rewritten within the reading group"
                    e = ring.get((w % RING, slot), (0.0, None, w))
                    assert e[2] == w, "ring slot overwritten or not written"
                    second.append((e[0], e[1]))
                elif md == 2:
                    second.append(qv[j])
                else:
                    second.append((0.0, None))  # the never-written ring column
            carried = st["prev"]
            st["prev"] = second
            if u <= 0 or u > n:
                writes.append((lane, 0.0, None))
                continue
            x = u if forward else n + 1 - u
            p = (x, y, z)
            vals = []
            for j in range(3):
                a, bb = neighbours(y, z, x, j)
                vals.append((checked(a, carried[j]), checked(bb, second[j])))
            own = (x - 1, y, z) if forward else (x + 1, y, z)
            v1 = checked(own, (st["v1"], st["v1p"]))
            slotv = pw[(prow(tau), lane)]
            assert slotv[1] == p
            if forward:
                Lp = lambda d: Ls[d][point_id(*p)]
                # d: w s se bnw bn bc be = 0..6 (the paper's D_l)
                acc = slotv[0]
                acc -= Lp(1) * vals[0][0] + Lp(2) * vals[0][1] + Lp(3) * vals[2][0] + Lp(4) * vals[2][1]
                acc -= Lp(5) * vals[1][0] + Lp(6) * vals[1][1] + Lp(0) * v1
            else:
                acc = Dinv[point_id(*p)] * slotv[0]

                def Lq(d, q):  # L~^{p-d}_d at q = p - d
                    return Ls[d][point_id(*q)] if interior(q) else 0.0
                a0, b0 = neighbours(y, z, x, 0)
                a1, b1 = neighbours(y, z, x, 1)
                a2, b2 = neighbours(y, z, x, 2)
                acc -= Lq(1, a0) * vals[0][0] + Lq(5, a1) * vals[1][0] + Lq(3, a2) * vals[2][0]
                acc -= Lq(2, b0) * vals[0][1] + Lq(6, b1) * vals[1][1] + Lq(4, b2) * vals[2][1]
                acc -= Lq(0, own) * v1
            writes.append((lane, acc, p))
        for lane, acc, p in writes:
            ring[(tau % RING, lane)] = (acc, p, tau)
            state[lane]["v1"], state[lane]["v1p"] = acc, p
            pending.append((tau, lane, acc, p))
        if tau % 4 == 3:  # the four-step block's results over their inputs
            for s_, lane, acc, p in pending:
                key = (prow(s_), lane)
                assert pw[key][1] == p, "result written to another point's slot"
                pw[key] = [acc, p, tag, s_]
            pending = []
    assert not pending


@pytest.mark.parametrize("level,lanes,quantum", [(3, 0, 0), (4, 0, 0), (5, 0, 0), (5, 24, 0), (6, 48, 0), (6, 0, 0),
                                                (4, 0, 2), (5, 24, 4), (6, 48, 2), (6, 40, 4), (6, 700, 4)])
def test_emulated_schedule_sweep_equals_the_oracle(g, orc, level, lanes, quantum):
    """Level 3-6 on the kernels' 384 lanes and on few lanes (which forces
    long delays and far producers read from global memory), with the
    kernels' start quantum and with quanta 2 and 4 (the level-7 and level-8
    kernels' row padding, switch steps and barrier groups), and on 700 lanes
    (lane numbers of a two-CTA cluster): the emulated sweep equals the
    oracle's sweep to FP64 rounding."""
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
    r_, _ = orc.residual(pr.A, N, x0, b)
    T, ln, ent_f, off = g.packed_schedule(level, True, lanes, quantum)
    _, _, ent_b, off_b = g.packed_schedule(level, False, lanes, quantum)
    assert np.array_equal(off, off_b)
    rows_f = [[decode(ent_f[e]) for e in range(off[l], off[l + 1])] for l in range(ln)]
    rows_b = [[decode(ent_b[e]) for e in range(off[l], off[l + 1])] for l in range(ln)]
    # the packed array: r of every point at (forward step of the point, lane), 0 elsewhere
    pw = {(s_, l): [0.0, None, "r", -1] for s_ in range(T) for l in range(ln)}
    for l in range(ln):
        for r in rows_f[l]:
            for x in range(1, r["n"] + 1):
                pw[(r["lo"] + x - 1, l)] = [r_[orc.index(N, x, r["y"], r["z"])], (x, r["y"], r["z"]), "r", -1]
    B = quantum or quantum_of(level)
    emulate_pass(N, T, ln, rows_f, True, Ls, Dinv, point_id, pw, B)
    emulate_pass(N, T, ln, rows_b, False, Ls, Dinv, point_id, pw, B)
    x = x0.copy()
    for (s_, l), (v, p, tag, _) in pw.items():
        assert tag == "b"
        if p is None:
            assert v == 0.0
            continue
        x[orc.index(N, *p)] += v
    assert np.abs(x - want).max() <= 1e-12 * np.abs(want).max()
    far = sum(int(mode(int(c) & 0xffffffff) == 2) for e in np.concatenate([ent_f, ent_b]) for c in e[5:8])
    if 0 < lanes < LANES and level >= 6:
        assert far > 0  # few lanes: the run exercised the global-memory path


@pytest.mark.parametrize("level", [5, 6, 7, 8])
def test_schedule_covers_every_row_once(g, orc, level):
    """Each interior row appears once per pass on the same lane; a lane's rows
    follow one another with a step without a point after every row and the
    coefficient-copy distance the kernel relies on, in both passes; switch
    steps sit on the level's quantum and producers are at least quantum + 1
    steps ahead; the backward pass is the forward one reversed in time; the
    entries' ring words, far bits and row coordinates are the ones the kernel
    would compute from the producer codes."""
    N = 2 ** level
    q = quantum_of(level)
    T, ln, ef, off = g.packed_schedule(level, True)
    _, _, eb, _ = g.packed_schedule(level, False)
    assert T % BLOCK == 0 and ln == lanes_of(level)
    ring_max = min(RING - 1, RING + 1 - q)
    RW = ln + 8  # ring row: every lane's column, then column ln that nothing writes
    for fwd, ent in ((True, ef), (False, eb)):
        rows = [decode(e) for e in ent]
        assert len({(r["y"], r["z"]) for r in rows}) == len(rows) == (N - 3) * (N - 2) // 2
        for r in rows:
            assert r["n"] == N - 1 - r["y"] - r["z"] and 1 <= r["lo"] - r["sw"] <= q and r["sw"] % q == q - 1
            assert r["lo"] + r["n"] <= T and r["sw"] >= 0
            K = N - r["y"] - r["z"]
            x_sw = 0 if fwd else r["n"] + r["lo"] - r["sw"]
            assert r["tt0"] == np.float32((2 * x_sw - K) * (0.5 / N))
            tau0 = r["sw"] & ~(BLOCK - 1)
            for j, c in enumerate(r["codes"]):
                md = mode(c)
                lane_p, k0 = lane_k0(c)
                if md == 1:
                    assert q + 1 <= k0 <= ring_max
                    assert r["R"][j] == ((tau0 + 1 - k0) % RING) * RW + lane_p
                else:
                    assert r["R"][j] == ln and (k0 > ring_max if md == 2 else k0 == 0)
                assert ((r["gm"] >> j) & 1) == (md == 2)
        for l in range(ln):
            prev = None
            for e in ent[off[l]:off[l + 1]]:
                r = decode(e)
                if prev is not None:
                    assert r["sw"] >= prev["lo"] + prev["n"]          # the step after a row has no point
                    assert r["sw"] >= prev["sw"] + PRE + 1            # the stage is free for the copy
                prev = r
    for l in range(ln):
        fw = [decode(e) for e in ef[off[l]:off[l + 1]]]
        bw = [decode(e) for e in eb[off[l]:off[l + 1]]]
        assert [(r["y"], r["z"]) for r in bw] == [(r["y"], r["z"]) for r in reversed(fw)]
        assert [r["lo"] for r in bw] == [T - r["lo"] - r["n"] for r in reversed(fw)]
