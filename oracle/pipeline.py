"""Buffer-hazard rule of the Section IV pipeline, as a checker over issued schedules.

TEST INFRASTRUCTURE ONLY.

Section IV: the five stages S(b_j), S(a_i), S(c_ij), DGEMM, R(c_ij) run on
streams ordered by recorded/waited events, and data in a device buffer must
not be overwritten until the kernels that operate on it have completed.  A
kernel must also see the data it was scheduled for (its inputs copied in
before it starts) and R(c_ij) must copy out the block the kernel produced.

A schedule is the list of operations in host issue order.  Each operation is a
dict with
    kind    'h2d' | 'kernel' | 'd2h' | 'record' | 'wait'
    stream  integer stream id
    writes  list of (slot, tag)  -- device slots written and the datum they then hold
    reads   list of (slot, tag)  -- device slots read and the datum expected there
    event   event id (record / wait)
CUDA stream semantics: operations of one stream run in issue order; a wait on
event E orders every later operation of its stream after everything issued on
the recording stream before the most recent record of E issued earlier.

check(schedule, initial) returns a list of violation strings (empty when the
rule holds for every execution the stream/event order allows); `initial` lists
slot contents left on the device by an earlier call (Section IV's nsteps
invocations, where C blocks stay resident between calls):
  * a read is not preceded (happens-before) by a write of the expected tag to
    that slot, or another write to the slot may fall between them;
  * two writes of one slot are unordered;
  * a write is unordered with a read of the same slot.
"""


def _vector_clocks(schedule):
    streams = sorted({op["stream"] for op in schedule})
    sidx = {s: i for i, s in enumerate(streams)}
    n = len(streams)
    cur = {s: [0] * n for s in streams}     # clock of each stream's tail
    last_record = {}                         # event -> clock captured at its latest record
    clocks = []
    for pos, op in enumerate(schedule):
        s = op["stream"]
        vc = list(cur[s])
        if op["kind"] == "wait":
            ev = op["event"]
            if ev not in last_record:
                raise ValueError("wait on event %r before any record (op %d)" % (ev, pos))
            rec = last_record[ev]
            vc = [max(a, b) for a, b in zip(vc, rec)]
        vc[sidx[s]] += 1
        cur[s] = vc
        if op["kind"] == "record":
            last_record[op["event"]] = list(vc)
        clocks.append(vc)
    return clocks


def _hb(a, b):
    """a happens-before b (vector clocks; a != b)."""
    return all(x <= y for x, y in zip(a, b)) and a != b


def check(schedule, initial=()):
    """initial: (slot, tag) pairs held by device slots before the schedule
    starts (data a previous call left resident); they happen before every op."""
    raw = _vector_clocks(schedule)
    zero = [0] * (len(raw[0]) if raw else 0)

    class _Clocks:
        def __getitem__(self, pos):
            return zero if pos < 0 else raw[pos]
    clocks = _Clocks()
    violations = []
    writes = {slot: [(-1, tag)] for slot, tag in initial}   # slot -> list of (pos, tag)
    reads = {}    # slot -> list of (pos, tag)
    for pos, op in enumerate(schedule):
        for slot, tag in op.get("writes", []):
            writes.setdefault(slot, []).append((pos, tag))
        for slot, tag in op.get("reads", []):
            reads.setdefault(slot, []).append((pos, tag))
    for slot, ws in writes.items():
        for x in range(len(ws)):
            for y in range(x + 1, len(ws)):
                p, q = ws[x][0], ws[y][0]
                if not (_hb(clocks[p], clocks[q]) or _hb(clocks[q], clocks[p])):
                    violations.append("unordered writes to %r at ops %d and %d" % (slot, p, q))
    for slot, rs in reads.items():
        ws = writes.get(slot, [])
        for rpos, tag in rs:
            before = [w for w in ws if _hb(clocks[w[0]], clocks[rpos])]
            if not before:
                violations.append("read of %r (%r) at op %d has no prior write" % (slot, tag, rpos))
                continue
            # the latest write that happens-before the read (writes are totally ordered)
            last = before[0]
            for w in before[1:]:
                if _hb(clocks[last[0]], clocks[w[0]]):
                    last = w
            if last[1] != tag:
                violations.append("read of %r at op %d expects %r, finds %r (op %d)"
                                  % (slot, rpos, tag, last[1], last[0]))
            for w in ws:
                if w is last or w in before or w[0] == rpos:
                    continue  # an operation's own writes land after its reads
                if not _hb(clocks[rpos], clocks[w[0]]):
                    violations.append("write of %r at op %d may overwrite it before the read at op %d"
                                      % (slot, w[0], rpos))
    return violations


def final_host_writes(schedule):
    """(slot, tag) of every d2h operation, in issue order (what reaches the host)."""
    out = []
    for op in schedule:
        if op["kind"] == "d2h":
            out.extend(op.get("reads", []))
    return out
