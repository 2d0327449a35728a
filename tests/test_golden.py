"""The figures the paper prints (tests/golden/paper_figures.txt): every line
parses and cites the section it comes from."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_figures.txt")


def test_paper_figures_parse_and_cite():
    rows = [line.split("|") for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    assert rows
    for r in rows:
        assert len(r) == 4, r
        name, value, unit, where = (x.strip() for x in r)
        assert name and value and unit
        assert where.startswith("Sec. "), r
    figs = {r[0].strip(): r[1].strip() for r in rows}
    assert float(figs["collide_speedup_two_loop_over_fused"]) == 2.5
    assert int(figs["particles_of_the_speedup_measurement"]) == 131072
