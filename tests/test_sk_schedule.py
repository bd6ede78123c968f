"""Race check of the blocked SK sweep's launch schedule (`SkModel::sweep` in
paper_1906_11195_gb300/csrc/sg_sk.cu), on the CPU.

The schedule under test is the library's own: `sg_sk_blocked_schedule` returns the operations
`SkModel::sweep` issues (it runs them from the same list), with their streams, events and row
skip ranges.  Each kernel's data is fixed by what the kernel does: the K* table kernel writes the
table; in-block(b) reads the table, its rows of H and the spins and flips of blocks b - 1 and b,
and writes its rows of H, block b's spins, flips and spin changes D; the field update of block b
reads D_b and writes the rows it updates.  Happens-before follows CUDA's rules: stream order,
and a stream wait on an event orders after the event's latest record issued before the wait.
Every pair of kernels touching the same data (a row tile of the fields H, a block's spin changes
D, spins and flip masks, the K* table), at least one of them writing, must be ordered, over
consecutive sweeps, for every block size and for sizes that leave a ragged last block.  A
restatement of the schedule from the host code's rules (`build_schedule`) must agree with the
library's and carries the planted mistakes.
"""
import itertools

import pytest

TILE = 128


def build_schedule(n, B, sweeps):
    """Ops as dicts {stream, kind, reads, writes}; waits as {stream, wait: event}; records as
    {stream, record: event}, in host issue order."""
    Np = -(-n // B) * B  # padded size: a multiple of B (and of 128 for B >= 128)
    ntiles, nblocks = Np // TILE, -(-n // B)
    ops = []

    def tiles_of_block(b):
        return set(range(b * B // TILE, min(ntiles, (b * B + B) // TILE)))

    for _ in range(sweeps):
        ops.append({"stream": "main", "kind": "kstar", "reads": set(),
                    "writes": {("kst", "all")}})
        pending = [False, False]
        for b in range(nblocks):
            if pending[b & 1]:
                ops.append({"stream": "main", "wait": ("side_done", b & 1)})
                pending[b & 1] = False
            reads = {("kst", "all")} | {("H", t) for t in tiles_of_block(b)}
            writes = {("H", t) for t in tiles_of_block(b)} | {("S", b), ("flips", b), ("D", b)}
            if b > 0:
                reads |= {("S", b - 1), ("flips", b - 1)}
            reads |= {("S", b)}
            ops.append({"stream": "main", "kind": f"inblock{b}", "reads": reads, "writes": writes})
            skip = set()
            if b + 1 < nblocks:
                skip = set(range((b * B + B) // TILE, min(ntiles, (b * B + 2 * B) // TILE)))
            rows = {("H", t) for t in range(ntiles) if t not in skip}
            ops.append({"stream": "main", "record": ("inblock_done", b & 1)})
            ops.append({"stream": "side", "wait": ("inblock_done", b & 1)})
            ops.append({"stream": "side", "kind": f"field{b}", "reads": {("D", b)} | rows,
                        "writes": rows})
            ops.append({"stream": "side", "record": ("side_done", b & 1)})
            pending[b & 1] = True
        for k in range(2):
            if pending[k]:
                ops.append({"stream": "main", "wait": ("side_done", k)})
    return ops


def happens_before(ops):
    """Transitive closure over kernels: stream order plus event record -> wait edges."""
    n = len(ops)
    pred = [set() for _ in range(n)]
    last_in_stream = {}
    last_record = {}
    for i, op in enumerate(ops):
        s = op["stream"]
        if s in last_in_stream:
            pred[i].add(last_in_stream[s])
        last_in_stream[s] = i
        if "record" in op:
            last_record[op["record"]] = i
        if "wait" in op and op["wait"] in last_record:
            pred[i].add(last_record[op["wait"]])
    before = [set() for _ in range(n)]
    for i in range(n):
        for p in pred[i]:
            before[i] |= before[p] | {p}
    return before


def races(ops):
    before = happens_before(ops)
    kernels = [i for i, op in enumerate(ops) if "kind" in op]
    found = []
    for i, j in itertools.combinations(kernels, 2):
        a, b = ops[i], ops[j]
        conflict = (a["writes"] & (b["reads"] | b["writes"])) or (b["writes"] & a["reads"])
        if conflict and i not in before[j] and j not in before[i]:
            found.append((a["kind"], b["kind"], sorted(conflict)[:3]))
    return found


TILE_OPS = {0: "kstar", 1: "inblock", 2: "field_all", 3: "field_rows", 4: "record", 5: "wait"}


@pytest.fixture(scope="module")
def sg():
    from paper_1906_11195_gb300 import _build
    _build.build()
    import paper_1906_11195_gb300 as m
    return m


def recorded_schedule(sg, n, B, sweeps):
    """The library's schedule of `sweeps` consecutive sweeps, as ops with their data."""
    unit = max(128, B)
    Np = -(-n // unit) * unit
    ntiles = Np // TILE
    ops = []
    streams = ("main", "side")
    events = (("inblock_done", 0), ("inblock_done", 1), ("side_done", 0), ("side_done", 1))

    def tiles_of_block(b):
        lo, hi = b * B, b * B + B
        return set(range(lo // TILE, min(ntiles, -(-hi // TILE))))

    for _ in range(sweeps):
        for op, st, b, s0, s1, ev in sg.sg_sk_blocked_schedule(n, B).tolist():
            stream = streams[st]
            kind = TILE_OPS[op]
            if kind == "kstar":
                ops.append({"stream": stream, "kind": "kstar", "reads": set(), "writes": {("kst", "all")}})
            elif kind == "inblock":
                rows = {("H", t) for t in tiles_of_block(b)}
                reads = {("kst", "all"), ("S", b)} | rows
                if b > 0:
                    reads |= {("S", b - 1), ("flips", b - 1)}
                ops.append({"stream": stream, "kind": f"inblock{b}", "reads": reads,
                            "writes": rows | {("S", b), ("flips", b), ("D", b)}})
            elif kind in ("field_all", "field_rows"):
                keep = [t for t in range(ntiles) if kind == "field_all" or not (s0 <= t < s1)]
                rows = {("H", t) for t in keep}
                ops.append({"stream": stream, "kind": f"field{b}", "reads": {("D", b)} | rows,
                            "writes": rows})
            elif kind == "record":
                ops.append({"stream": stream, "record": events[ev]})
            else:
                ops.append({"stream": stream, "wait": events[ev]})
    return ops


@pytest.mark.parametrize("B", [64, 128, 256, 512])
@pytest.mark.parametrize("n", [1024, 1000, 2176, 4096])
def test_blocked_sweep_schedule_has_no_race(sg, n, B):
    if n < B:
        pytest.skip("fewer spins than one block")
    assert races(recorded_schedule(sg, n, B, sweeps=2)) == []


@pytest.mark.parametrize("B", [128, 256, 512])
@pytest.mark.parametrize("n", [1024, 1000, 2176])
def test_restated_schedule_is_the_librarys(sg, n, B):
    def shape(ops):
        return [(op["stream"], op.get("kind"), op.get("record"), op.get("wait"),
                 sorted(op.get("writes", ()))) for op in ops]
    assert shape(recorded_schedule(sg, n, B, sweeps=2)) == shape(build_schedule(n, B, sweeps=2))


def test_race_check_catches_a_wrong_skip_range():
    # the field update of block b also touching block b+1's rows races with in-block(b+1)
    ops = build_schedule(1024, 256, sweeps=1)
    for op in ops:
        if op.get("kind", "").startswith("field"):
            op["writes"] = op["reads"] = {("H", t) for t in range(1024 // TILE)} | {("D", int(op["kind"][5:]))}
    assert any(a.startswith("inblock") or b.startswith("inblock") for a, b, _ in races(ops))


def test_race_check_catches_a_missing_join():
    # in-block(b+2) not waiting for field(b): field(b) writes block b+2's rows
    ops = [op for op in build_schedule(1024, 128, sweeps=1)
           if not (op.get("wait") == ("side_done", 0) and op["stream"] == "main")]
    assert races(ops)
