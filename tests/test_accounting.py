"""The bench's byte/flop accounting reproduces the figures printed in Sec. 2."""
import json
import os

from paper_1010_4782_gb300 import accounting

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cost_model.json")


def test_per_site_figures_match_the_paper():
    g = json.load(open(GOLDEN))
    assert accounting.paper_bytes_per_site(naik=False) == g["bytes_per_site"]
    assert accounting.flops_per_site(naik=False) == g["flops_per_site"]


def test_lattice_totals_match_the_paper():
    g = json.load(open(GOLDEN))
    flops, paper_bytes, _ = accounting.dslash_totals(tuple(g["lattice"]), naik=False)
    # the paper prints one significant digit (0.607 G -> 0.6, 1.669 GB -> 1.6)
    assert int(flops / 1e8) / 10 == g["total_gflop_printed"]
    assert int(paper_bytes / 1e8) / 10 == g["total_gbyte_printed"]


def test_compulsory_and_naik_figures():
    assert accounting.compulsory_bytes_per_site(False) == 1248
    assert accounting.compulsory_bytes_per_site(True) == 2400
    assert accounting.compulsory_bytes_per_site(True, long_entries=6) == 2016  # 8 x 144 + 8 x 96 + 96
    assert accounting.compulsory_bytes_per_site(False, long_entries=6) == 1248
    assert accounting.paper_bytes_per_site(True) == 3120
    assert accounting.flops_per_site(True) == 1152
    assert accounting.compulsory_bytes_per_site(True, elem_bytes=4) == 1200
    assert accounting.compulsory_bytes_per_site(False, elem_bytes=2) == 312
    assert accounting.multi_rhs_bytes_per_site(16) == 1920
    assert accounting.multi_rhs_bytes_per_site(1) == 1200  # one RHS: the FP32 single-RHS figure
    assert accounting.multi_rhs_bytes_per_site(8, naik=False) == 8 * 72 + 8 * 48


def test_fma_count_is_half_the_papers_flop_count():
    """Every real multiplication of the SU(3) x vector products is fused with an addition, so
    the paper's 576 flops per one-hop site (Sec. 2) are 288 FMAs; 576 with the Naik hops."""
    g = json.load(open(GOLDEN))
    assert 2 * accounting.fma_per_site(False) == g["flops_per_site"]
    assert accounting.fma_per_site(True) == 576
