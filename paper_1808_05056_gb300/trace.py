"""Summaries of the pipeline timeline recorded with ``OOC_TRACE=<file>``.

With that variable set, every out-of-core call appends a ``# call ...`` header and one CSV line
per H2D copy, kernel and D2H copy: ``kind,stream,i,j,kc,bytes,host_ms,start_ms,end_ms``, the
times in ms from the call's first event, taken with CUDA events on the op's own stream (the
timeline of Section IV's Fig. 3: copies in both directions overlapping the kernels).

    python -m paper_1808_05056_gb300.trace FILE [--call N] [--json]

prints per call: its span; each stream's busy time (the union of its ops' intervals); how much
of the copy time ran while a kernel was running; and the kernel stream's idle time inside the
span, split into fill (before the first kernel), drain (after the last) and gaps between
kernels.  Host-side only; no GPU needed.
"""
import argparse
import json
import sys

KINDS = ("h2d", "kernel", "d2h")


def parse(path):
    """The calls of a trace file: [{"header": {...}, "ops": [(kind, stream, i, j, kc, bytes, host_ms,
    start_ms, end_ms), ...]}] (lines of other tools' traces in the same file are skipped)."""
    calls = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# call"):
                hdr = {}
                for tok in line[len("# call"):].split():
                    k, _, v = tok.partition("=")
                    hdr[k] = int(v)
                calls.append({"header": hdr, "ops": []})
                continue
            parts = line.split(",")
            if not calls or len(parts) != 9 or parts[0] not in KINDS:
                continue
            kind = parts[0]
            stream, i, j, kc = (int(x) for x in parts[1:5])
            nbytes, host, t0, t1 = (float(x) for x in parts[5:9])
            calls[-1]["ops"].append((kind, stream, i, j, kc, nbytes, host, t0, t1))
    return calls


def union(intervals):
    """Disjoint sorted union of [a, b) intervals."""
    out = []
    for a, b in sorted(intervals):
        if b <= a:
            continue
        if out and a <= out[-1][1]:
            out[-1][1] = max(out[-1][1], b)
        else:
            out.append([a, b])
    return [tuple(x) for x in out]


def length(u):
    return sum(b - a for a, b in u)


def intersect_length(u, v):
    """Measure of the intersection of two disjoint sorted unions."""
    total, p, q = 0.0, 0, 0
    while p < len(u) and q < len(v):
        a, b = max(u[p][0], v[q][0]), min(u[p][1], v[q][1])
        if b > a:
            total += b - a
        if u[p][1] < v[q][1]:
            p += 1
        else:
            q += 1
    return total


def summarize(call):
    """Overlap figures of one call (times in ms, bytes in bytes, rates in GB/s)."""
    ops = call["ops"]
    by = {k: [(o[7], o[8]) for o in ops if o[0] == k] for k in KINDS}
    u = {k: union(v) for k, v in by.items()}
    t_begin = min((o[7] for o in ops), default=0.0)
    t_end = max((o[8] for o in ops), default=0.0)
    span = t_end - t_begin
    busy = {k: length(u[k]) for k in KINDS}
    kern = u["kernel"]
    fill = (kern[0][0] - t_begin) if kern else span
    drain = (t_end - kern[-1][1]) if kern else 0.0
    gaps = sum(b[0] - a[1] for a, b in zip(kern, kern[1:]))
    out = {"span_ms": span, "ops": {k: len(by[k]) for k in KINDS}, "busy_ms": busy,
           "kernel_busy_frac": busy["kernel"] / span if span > 0 else None,
           "kernel_idle_ms": {"fill": fill, "gaps": gaps, "drain": drain}}
    for k in ("h2d", "d2h"):
        nbytes = sum(o[5] for o in ops if o[0] == k)
        hidden = intersect_length(u[k], kern)
        out[k] = {"bytes": nbytes, "busy_ms": busy[k],
                  "gbps_while_busy": nbytes / (busy[k] * 1e6) if busy[k] > 0 else None,
                  "under_kernels_ms": hidden,
                  "under_kernels_frac": hidden / busy[k] if busy[k] > 0 else None}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("file")
    ap.add_argument("--call", type=int, default=None, help="only this call (0-based)")
    ap.add_argument("--json", action="store_true", help="one JSON object per call")
    a = ap.parse_args(argv)
    calls = parse(a.file)
    picks = range(len(calls)) if a.call is None else [a.call]
    for n in picks:
        c = calls[n]
        s = summarize(c)
        if a.json:
            print(json.dumps({"call": n, "header": c["header"], **s}))
            continue
        h = c["header"]
        print("call %d: M=%s N=%s K=%s mb=%s nb=%s kb=%s" % (n, h.get("M"), h.get("N"), h.get("K"), h.get("mb"),
                                                           h.get("nb"), h.get("kb")))
        print("  span %.1f ms; kernels %d, busy %.1f ms (%.1f %% of the span)" % (
            s["span_ms"], s["ops"]["kernel"], s["busy_ms"]["kernel"], 100 * (s["kernel_busy_frac"] or 0)))
        ki = s["kernel_idle_ms"]
        print("  kernel stream idle: fill %.1f ms, gaps %.1f ms, drain %.1f ms" % (ki["fill"], ki["gaps"],
                                                                                 ki["drain"]))
        for k in ("h2d", "d2h"):
            d = s[k]
            print("  %s: %d copies, %.2f GB, busy %.1f ms (%.0f GB/s while busy), %.1f %% under kernels" % (
                k, s["ops"][k], d["bytes"] / 1e9, d["busy_ms"], d["gbps_while_busy"] or 0,
                100 * (d["under_kernels_frac"] or 0)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
