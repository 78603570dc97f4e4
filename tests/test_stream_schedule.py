"""The streamed level programs as the host builds them (no GPU): an independent parser
of the chunk format checks that every barrier-free stretch is race-free and that the
records cover the program.

Within a stretch the consumer threads run without synchronising, so a record on thread
t may read a slot only if no other thread wrote it in the stretch, and may overwrite a
slot only if no other thread read or wrote it there. The check reads the raw chunks;
only the segment barrier bit separates stretches (chunk boundaries do not synchronise
the consumer group). A replay with hashed values then runs every stretch thread by
thread in two opposite thread orders and compares with the plain wave order (the
level-by-level semantics of Sec. 3.1)."""
import struct

import numpy as np
import pytest

from paper_2303_08881_gb300 import problems as P

CASES = {
    "poisson64": lambda: P.make_workload("poisson2d_64_p4"),
    "aniso2d_ragged": lambda: P.aniso2d_boxes(70, 3, seed=1),
    "aniso2d_128box": lambda: P.aniso2d_boxes(256, 2, seed=7),
    "conv3d": lambda: P.convdiff3d_boxes(14, 2, seed=2),
    "cuts3d": lambda: P.aniso3d_cuts(20, ncuts=(2, 2, 1), seed=3),
    "rand": lambda: P.randsparse(3000, 8, mean_k=4.0, seed=4),
    "p1": lambda: P.aniso2d_boxes(30, 1, seed=5),
    "dense_rows": lambda: P.randsparse(1500, 2, mean_k=24.0, seed=6),
}
CFGS = [
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0"),
    dict(variant="schur", factor_B="ilut", factor_S="milu0", ilut_tau=1e-3, ilut_p=10),
    dict(variant="rap", factor_B="ilu0", factor_S="milu0"),
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", local_order="rcm"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", local_order="rcm"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", fill_level=2),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", pc_precision="bf16"),
    dict(variant="rap", factor_B="ilu0", factor_S="milu0", pc_precision="bf16"),
]
SKIP = 1 << 31
BARRIER = 1 << 31
SCAN = 1 << 30        # segment word 1: a scan segment
EACH = 1 << 29        # segment word 1: a barrier after every wave
LINK_COL = 1 << 30    # record head: linked to the previous row of the warp through col[0]
LINK_SELF = 1 << 29   # record head: linked through the own slot


@pytest.fixture(scope="module")
def ilu():
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as m
    return m


def _al(x, a):
    return (x + a - 1) // a * a


def parse(st):
    """Per subdomain: a list of stretches (the rows between two barriers); a stretch is a
    list of waves; a wave is a list of (thread, write_slot, [read slots], link) with skip
    records left out, link = None in plain waves and 0 / "col" / "self" in scan waves.
    Checks the geometry and the padding of every record."""
    blob, ch0, chunk, rw, vb = st["blob"].tobytes(), st["ch0"], st["chunk"], st["rw"], st["val_bytes"]
    xb = st["x_bytes"]  # element size of the working vector and of dinv
    col_off = 2 * xb
    rec_bytes = _al(_al(2 * xb + 4 * rw, vb) + rw * vb, 16)
    subs = []
    for s in range(len(ch0) - 1):
        stretches, cur = [], []
        for c in range(ch0[s], ch0[s + 1]):
            cb = c * chunk
            nseg = struct.unpack_from("<I", blob, cb)[0]
            end = 16 + _al(8 * nseg, 16)
            for g in range(nseg):
                w0, w1 = struct.unpack_from("<II", blob, cb + 16 + 8 * g)
                off, width, nw = (w0 & 0xFFFF) * 16, (w0 >> 16) & 0x1FF, w1 & 0xFFFF
                assert off >= end and off + nw * width * rec_bytes <= chunk and 1 <= width <= st["threads"]
                scan = bool(w1 & SCAN)
                assert not scan or width % 32 == 0
                end = off + nw * width * rec_bytes
                for w in range(nw):
                    wave = []
                    for t in range(width):
                        rb = cb + off + (w * width + t) * rec_bytes
                        head = struct.unpack_from("<I", blob, rb)[0]
                        cols = struct.unpack_from(f"<{rw}I", blob, rb + col_off)
                        if head & SKIP:
                            assert head == SKIP and not any(cols)
                            continue
                        n, row = (head >> 24) & 0x1F, head & 0xFFFFFF  # the head holds the row's index
                        link = ("col" if head & LINK_COL else "self" if head & LINK_SELF else 0) if scan else None
                        assert scan or not head & (LINK_COL | LINK_SELF), "links only in scan segments"
                        assert not (head & LINK_COL and head & LINK_SELF) and (link != "col" or n >= 1)
                        assert n <= rw and all(x % xb == 0 for x in cols)
                        assert all(x == row * xb for x in cols[n:]), "unused entries read the row's own slot"
                        wave.append((t, row, [x // xb for x in cols[:n]], link))
                    cur.append(wave)
                    if w1 & EACH:
                        assert not scan and not w1 & BARRIER
                        stretches.append(cur)
                        cur = []
                if w1 & BARRIER:
                    stretches.append(cur)
                    cur = []
        if cur:
            stretches.append(cur)
        subs.append(stretches)
    return subs


def _is_scan(stretch):
    kinds = {r[3] is not None for wave in stretch for r in wave}
    assert len(kinds) <= 1, "a stretch mixes scan and plain waves"
    return kinds == {True}


def hazards(stretches):
    """Plain stretches: a thread may read a slot only if no other thread wrote it in the
    stretch, and overwrite one only if no other thread read or wrote it there. Scan
    stretches: the executor is the warp, in (wave, lane) order; a value written in the same
    wave may be read only through the link (one lane below, via col[0] or the own slot), a
    link must name exactly that writer, and no slot is shared between warps."""
    bad = 0
    for stretch in stretches:
        scan = _is_scan(stretch)
        writer, readers = {}, {}
        for wi, wave in enumerate(stretch):
            for t, w, cols, link in wave:
                ex = t // 32 if scan else t
                lane = t % 32
                for qi, c in enumerate(list(cols) + [w]):
                    wr = writer.get(c)
                    if wr is not None:
                        if wr[0] != ex:
                            bad += 1
                        elif scan and wr[1] == wi:
                            via = "self" if c == w and qi == len(cols) else ("col" if qi == 0 else None)
                            if not (link == via and wr[2] == lane - 1 and lane > 0):
                                bad += 1
                    readers.setdefault(c, set()).add(ex)
                if scan and link and lane > 0:
                    c = cols[0] if link == "col" else w
                    if writer.get(c) != (ex, wi, lane - 1):
                        bad += 1   # the link must name the previous row of the warp
                wr = writer.get(w)
                if (wr is not None and wr[0] != ex) or readers[w] - {ex}:
                    bad += 1
                writer[w] = (ex, wi, lane)
    return bad


def replay(stretches, order):
    """The rows with hashed values, stretch after stretch. "wave": wave by wave, threads in
    order; "up" / "down": each executor's rows in its own order (plain: thread, scan:
    warp), executors ascending / descending."""
    x = {}
    rid = 0
    for stretch in stretches:
        scan = _is_scan(stretch)
        recs = []
        for wi, wave in enumerate(stretch):
            for t, w, cols, link in wave:
                ex = t // 32 if scan else t
                recs.append((ex, wi, t, w, cols, rid))
                rid += 1
        if order == "wave":
            seq = recs
        else:
            sign = 1 if order == "up" else -1
            seq = sorted(recs, key=lambda r: (sign * r[0], r[1], r[2]))
        for ex, wi, t, w, cols, r in seq:
            x[w] = hash((x.get(w, ("in", w)), tuple(x.get(c, ("in", c)) for c in cols), r))
    return x


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: "-".join(map(str, c.values())))
def test_stretches_are_race_free(ilu, name, cfg):
    pr = CASES[name]()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, **cfg))
    sizes = h.sizes()
    progs = {"bj": ["bj"], "schur": ["fwd", "s", "bwd"], "rap": ["bj", "fwd", "bwd"]}[cfg["variant"]]
    for prog in progs:
        st = h.stream(prog)
        subs = parse(st)
        stats = h.stream_stats(prog)
        assert stats["threads"] == st["threads"]
        n_rec = sum(len(w) for stretches in subs for s in stretches for w in s)
        n_ent = sum(len(r[2]) for stretches in subs for s in stretches for w in s for r in w)
        n_scan = max(sum(len(s) for s in stretches if _is_scan(s)) for stretches in subs)
        assert n_scan == stats["max_scan_waves"] or prog == "bj"
        assert n_rec == stats["records"] - stats["skips"]
        if prog != "fwd":  # the forward stream also holds the S~ rows
            assert n_rec >= sizes[f"prog_{prog}"]["rows"]
            assert n_ent == sizes[f"prog_{prog}"]["entries"]
        assert max(len(s) for s in subs) - 1 <= stats["max_barriers"]
        assert stats["max_barriers"] <= stats["max_levels"] * (1 + (st["rw"] < 16))
        assert stats["max_steps"] <= stats["max_barriers"] + stats["max_scan_waves"]
        for s, stretches in enumerate(subs):
            assert hazards(stretches) == 0, (prog, s)
            ref = replay(stretches, "wave")
            assert replay(stretches, "up") == ref and replay(stretches, "down") == ref, (prog, s)
    h.close()


def test_interface_chains_run_as_warp_scans(ilu):
    """On 128 x 128 boxes of the 9-point problem the interface of a subdomain is a ring of
    chains (each row reads only the previous one of its side); the local Schur program and
    the interface part of the forward program run them as scan waves, 32 rows per warp and
    wave, with a handful of barriers where a plain level schedule needs one per level."""
    pr = P.aniso2d_boxes(256, 2, seed=0)
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True))
    st = h.stream_stats("s")
    assert st["max_levels"] > 250
    assert st["chain_sections"] == pr.p and st["max_barriers"] <= 10
    assert st["max_steps"] <= 48     # ~510 chained rows in <= 48 dependent steps
    fw = h.stream_stats("fwd")
    assert fw["chain_sections"] == pr.p and fw["max_scan_waves"] > 0
    h.close()


def test_planted_link_errors_are_detected():
    """the checker itself, on scan stretches: a read of a same-wave value that is not the
    link, a link to a row that is not the previous one, and two warps sharing a slot"""
    ok = [[[(0, 10, [], 0), (1, 11, [10], "col"), (2, 12, [11, 3], "col")]]]
    assert hazards(ok) == 0
    not_link = [[[(0, 10, [], 0), (1, 11, [], 0), (2, 12, [3, 10], "col")]]]  # reads lane 0's slot
    assert hazards(not_link) >= 1
    wrong_pred = [[[(0, 10, [], 0), (1, 11, [], 0), (2, 12, [10], "col")]]]   # linked to lane 0
    assert hazards(wrong_pred) >= 1
    self_link = [[[(0, 10, [3], 0), (1, 10, [4], "self")]]]                    # same slot, linked
    assert hazards(self_link) == 0
    cross_warp = [[[(0, 10, [], 0), (32, 13, [10], 0)]]]                      # warp 1 reads warp 0
    assert hazards(cross_warp) == 1
    later_wave = [[[(0, 10, [], 0)], [(1, 11, [10], 0)]]]                     # earlier wave, same warp
    assert hazards(later_wave) == 0


def test_planted_race_is_detected():
    """the checker itself: two threads touching one slot inside a stretch"""
    raw = [[[(0, 5, [1], None), (1, 6, [2], None)], [(1, 7, [5], None)]]]  # thread 1 reads slot 5 of thread 0
    assert hazards(raw) == 1
    ok = [[[(0, 5, [1], None), (1, 6, [2], None)]], [[(1, 7, [5], None)]]]  # a barrier in between
    assert hazards(ok) == 0
    war = [[[(0, 5, [3], None)], [(1, 3, [], None)]]]  # thread 1 overwrites what thread 0 read
    assert hazards(war) == 1
    a, b = replay(raw, "up"), replay(raw, "down")
    assert a != b or replay(raw, "wave") != a


def emulate(stretches):
    """The device's semantics on hashed values: a plain wave's rows run one after another
    (its threads are independent); in a scan wave each warp loads every operand of its 32
    rows before any of them stores, and a linked row (lane > 0) takes its predecessor's new
    value in place of the loaded one -- through col[0] or its own slot. A row's value
    hashes its slot and the (slot, value) pairs it read, so two schedules of one program
    give equal results exactly when every row sees the same inputs."""
    x = {}

    def val(c):
        return x.get(c, ("in", c))

    def row_hash(w, own, pairs):
        return hash((w, own, tuple(sorted(pairs))))

    for stretch in stretches:
        for wave in stretch:
            if not wave or wave[0][3] is None:
                for t, w, cols, link in wave:
                    x[w] = row_hash(w, val(w), [(c, val(c)) for c in cols])
                continue
            warps = {}
            for rec in wave:
                warps.setdefault(rec[0] // 32, []).append(rec)
            for u, recs in warps.items():
                snap = {c: val(c) for t, w, cols, link in recs for c in list(cols) + [w]}
                res = {}
                for t, w, cols, link in recs:
                    lane = t % 32
                    prev = res.get(lane - 1) if lane > 0 else None
                    own = prev[1] if (link == "self" and lane > 0) else snap[w]
                    pairs = [(c, prev[1] if (link == "col" and lane > 0 and qi == 0) else snap[c])
                             for qi, c in enumerate(cols)]
                    if link and lane > 0:
                        assert prev is not None, "a linked row needs its predecessor one lane below"
                    res[lane] = (w, row_hash(w, own, pairs))
                # the lanes store in one instruction: a slot written by two lanes of the wave
                # must be a row and its successor linked through that slot, whose lane stores
                lanes_of = {}
                for t, w, cols, link in recs:
                    lanes_of.setdefault(w, []).append((t % 32, link))
                for w, ls in lanes_of.items():
                    ls.sort()
                    for (la, _), (lb, lkb) in zip(ls, ls[1:]):
                        assert lb == la + 1 and lkb == "self", f"slot {w} stored by lanes {la} and {lb}"
                for lane, (w, v) in res.items():
                    if lanes_of[w][-1][0] == lane:
                        x[w] = v
    return x


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cfg", [c for c in CFGS if c["variant"] != "bj"], ids=lambda c: "-".join(map(str, c.values())))
def test_chain_schedule_computes_the_level_program(ilu, name, cfg):
    """Every subdomain program scheduled as chains (warp scans) computes, on the device's
    semantics, exactly what its level schedule computes: each row reads the same inputs."""
    pr = CASES[name]()
    res = {}
    for mode in ("levels", "chains"):
        h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, chain_sched=mode, **cfg))
        progs = ["fwd", "s"] if cfg["variant"] == "schur" else ["fwd"]
        res[mode] = {prog: [emulate(st) for st in parse(h.stream(prog))] for prog in progs}
        if mode == "chains":
            assert sum(h.stream_stats(p)["chain_sections"] for p in progs) > 0 or name in ("rand", "p1")
        h.close()
    for prog in res["levels"]:
        for s, (a, b) in enumerate(zip(res["levels"][prog], res["chains"][prog])):
            assert a == b, (prog, s)
