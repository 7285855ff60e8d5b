"""Text report of an analysis: one table per pattern with each code site's
count, wasted bytes, wasted time and that time as a share of the trace span,
then the optimisation-potential estimate (the paper's Sec. 7.6: predicted time
= total time minus the time of the eliminable transfers and allocations).

Sites are the integer site ids of the events; mapping them to source lines
needs the program's debug information and is left to the caller
(``site_names``).
"""

from __future__ import annotations

TITLES = {
    1: "Duplicate Target Data Transfer Analysis",
    2: "Round-Trip Target Data Transfer Analysis",
    3: "Repeated Device Memory Allocation Analysis",
    4: "Unused Device Memory Allocation Analysis",
    5: "Unused Target Data Transfer Analysis",
}


def _fmt_bytes(b: int) -> str:
    for unit in ("B", "KiB", "MiB", "GiB", "TiB"):
        if b < 1024 or unit == "TiB":
            return f"{b:.0f} {unit}" if unit == "B" else f"{b:.2f} {unit}"
        b /= 1024.0
    return f"{b} B"


def _fmt_ns(ns: int) -> str:
    if ns >= 1_000_000_000:
        return f"{ns / 1e9:.3f} s"
    if ns >= 1_000_000:
        return f"{ns / 1e6:.3f} ms"
    if ns >= 1_000:
        return f"{ns / 1e3:.3f} us"
    return f"{ns} ns"


def render(result: dict, site_names: dict | None = None, top: int = 10) -> str:
    """``result`` is ``Findings.to_host()`` (or the oracle's equivalent with
    keys status, summary, sites)."""
    s = result["summary"]
    span = max(1, s["trace_span_ns"])
    rows = result["sites"]
    lines = []
    for kind in range(1, 6):
        lines.append(f"=== OpenMP {TITLES[kind]} ===")
        lines.append(f"  findings: {s[f'count{kind}']}, wasted bytes: "
                     f"{_fmt_bytes(s[f'wasted_bytes{kind}'])}, wasted time: "
                     f"{_fmt_ns(s[f'wasted_ns{kind}'])} "
                     f"({100.0 * s[f'wasted_ns{kind}'] / span:.2f}% of the trace)")
        sel = [r for r in rows if int(r["kind"]) == kind]
        sel.sort(key=lambda r: -int(r["wasted_ns"]))
        if sel:
            lines.append(f"  {'time(%)':>8}  {'time':>12}  {'count':>10}  {'bytes':>12}  site")
            for r in sel[:top]:
                name = (site_names or {}).get(int(r["site"]), f"site {int(r['site'])}")
                lines.append(f"  {100.0 * int(r['wasted_ns']) / span:7.2f}%  "
                             f"{_fmt_ns(int(r['wasted_ns'])):>12}  {int(r['count']):>10}  "
                             f"{_fmt_bytes(int(r['wasted_bytes'])):>12}  {name}")
            if len(sel) > top:
                lines.append(f"  ... {len(sel) - top} more sites")
        lines.append("")
    den = s["speedup_den"]
    lines.append("=== Optimization Potential ===")
    lines.append(f"  trace span: {_fmt_ns(s['trace_span_ns'])}; eliminable time (union of "
                 f"wasted operations): {_fmt_ns(s['saved_ns'])}")
    if den:
        lines.append(f"  predicted time: {_fmt_ns(den)}; predicted speedup: "
                     f"{s['speedup_num'] / den:.3f}x")
    else:
        lines.append("  predicted speedup: unbounded (eliminable time covers the span)")
    return "\n".join(lines)
