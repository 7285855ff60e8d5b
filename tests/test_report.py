"""The text report (CPU: rendered from the oracle's result, whose layout the
GPU result shares)."""

from synth import traces


def test_report_listing2(orc):
    from paper_2601_12713_b300 import report

    b = traces.listing2(8)
    traces.fill_fp_from_content(b)
    r = orc.analyze(b.events)
    text = report.render({"summary": r.summary, "sites": r.sites, "status": r.status},
                         site_names={7: "listing2.c:4"})
    assert "Round-Trip Target Data Transfer Analysis" in text
    assert "findings: 7" in text and "listing2.c:4" in text
    span, saved = r.summary["trace_span_ns"], r.summary["saved_ns"]
    assert f"{span / (span - saved):.3f}x" in text
