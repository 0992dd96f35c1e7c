"""The flop model reproduces the FLOP columns of Tables 2 and 3 exactly."""

import os

from oracle import flops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_2_3_flop.txt")


def load():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            size, t2, t3 = line.split()
            rows.append((tuple(int(v) for v in size.split("x")), int(t2), int(t3)))
    return rows


def test_tables_2_and_3():
    rows = load()
    assert len(rows) == 5
    for block, t2, t3 in rows:
        assert flops.table2_flop(block) == t2
        assert flops.table3_flop(block) == t3


def test_per_site_counts():
    # 4^4 domains, n_sap = 4, n_jac = 4, chiral basis (168 flop for every hop)
    h = (168, 168, 168, 168)
    assert flops.f_in((4, 4, 4, 4), h) == 1608
    assert flops.f_out((4, 4, 4, 4), h) * 2 == 1797
    assert flops.D_FLOP_PER_SITE == 1320 + 504


def test_benchmark_restates_the_oracle_flop_model():
    """bench_configs restates the per-site flop model (it may not import the
    oracle outside the CPU-baseline leg); the two agree for cubic, elongated
    and the paper's own domain shapes."""
    import bench_configs
    h = (168, 168, 168, 168)
    for domain in ((4, 4, 4, 4), (16, 4, 2, 2), (8, 4, 4, 2), (16, 6, 4, 3), (16, 12, 8, 12)):
        for n_sap, n_jac in ((4, 2), (4, 4), (0, 1)):
            got = bench_configs._paper_flop_per_site_iter(domain, n_sap, n_jac, h)
            assert abs(got - flops.flop_per_site_iter(domain, n_sap, n_jac, h)) < 1e-9, (domain, n_sap, n_jac)


def test_sap_kernel_flop_count_uses_the_oracle_constants():
    """The roofline's flop count of the SAP block kernel (bench.sap_flop_per_site)
    is built from the oracle's per-site constants for 4^4 domains: f_in per
    A_cc application (n_jac Jacobi sweeps plus one for the residual update, 48
    for the update itself) and f_out for the surface term, averaged over the
    2 (n_sap + 1) launches of M_SAP."""
    import bench
    h = (168, 168, 168, 168)
    fi, fo = flops.f_in((4, 4, 4, 4), h), flops.f_out((4, 4, 4, 4), h)
    seq = []
    for sweep in range(bench.N_SAP + 1):
        for colour in (0, 1):
            surf = fo if not (sweep == 0 and colour == 0) else 0.0
            upd = fi + 48 if sweep < bench.N_SAP else 0.0
            seq.append(surf + bench.N_JAC * fi + upd)
    assert abs(bench.sap_flop_per_site() - sum(seq) / len(seq)) < 1e-9
    assert abs(bench.sap_flop_per_site() - 8565.45) < 1e-9


def test_dslash_roofline_constants():
    """The Dslash roofline counts 1824 flop (the oracle's) and 768 bytes per
    site: spinor in and out (2 x 96), four float32 links of 18 reals (288)
    and the two float32 clover blocks of 36 reals (288)."""
    import bench
    assert bench.D_FLOP_PER_SITE == flops.D_FLOP_PER_SITE
    assert bench.D_BYTES_PER_SITE == 2 * 24 * 4 + 4 * 18 * 4 + 2 * 36 * 4 == 768


def test_a64fx_node_rates_reproduce_table2_tflops():
    """The A64FX node rates the benchmark compares against (site-iterations
    per second of one node, from Table 2's times: four processes, each 500
    iterations on a block of two domains) times the paper-basis flop per
    site-iteration reproduce Table 2's TFLOPS column (0.8272 for 32x6x4x3,
    1.0839 for 32x6x4x6) to its printed digits."""
    import bench_configs
    for domain, tflops in (((16, 6, 4, 3), 0.8272), ((16, 6, 4, 6), 1.0839)):
        rate = bench_configs._a64fx_node_rate(domain)
        flop = flops.flop_per_site_iter(domain, 4, 2)
        assert abs(rate * flop / 1e12 - tflops) < 6e-5, (domain, rate * flop / 1e12)
