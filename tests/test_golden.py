"""The figures the paper prints (tests/golden/paper_figures.txt): every line
parses and cites the section it comes from, and the benchmark's Fig. 4 leg
runs at the paper's particle count and reports the paper's Collide speed-up
beside its own measurement."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "paper_figures.txt")


def test_paper_figures_parse_and_cite():
    rows = [line.split("|") for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    assert rows
    for r in rows:
        assert len(r) == 4, r
        name, value, unit, where = (x.strip() for x in r)
        assert name and value and unit
        assert where.startswith("Sec. "), r


def test_bench_fig4_leg_uses_the_papers_figures():
    sys.path.insert(0, ROOT)
    import bench
    pf = bench.paper_figures()
    assert pf["collide_speedup_two_loop_over_fused"]["value"] == 2.5
    assert pf["collide_speedup_two_loop_over_fused"]["where"].startswith("Sec. 5.2")
    assert bench.FIG4_PARTICLES == int(pf["particles_of_the_speedup_measurement"]["value"])
