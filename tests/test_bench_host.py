"""Host logic of bench.py, on the CPU: the extras switch and the oracle's stratified sample of
edge tasks (the CPU baseline's estimator), whose bands cover every arc of the roots that can hold
a k-clique."""
import numpy as np

import bench
import oracle
from paper_2112_10913_gb300 import graphgen as gg


def test_extras_switch():
    assert bench.extras_of(bench.parse([])) == set(bench.EXTRAS)
    assert bench.extras_of(bench.parse(["--extras", "none"])) == set()
    assert bench.extras_of(bench.parse(["--extras", "k7,serve,bogus"])) == {"k7", "serve"}


def test_stratified_sample_covers_the_eligible_roots(oracle_lib):
    g = gg.small_rmat(5, 3000, 12.0)
    dag, _ = bench.oracle_order(g)
    outdeg = np.diff(dag[0])
    for k in (4, 5):
        eligible = int(outdeg[outdeg >= k - 1].sum())
        # groups as large as the bands, within a generous budget: every band is sampled completely
        est, se, sampled, missing = bench.oracle_stratified(dag, g.n, k, budget_s=120, per=10 ** 6)
        assert sampled == eligible and not missing
        assert est >= 0.0 and se == 0.0  # a tiny graph may cost no more than the calls themselves
        # the default plan: every band sampled, round-robin from the heaviest down
        est2, se2, sampled2, missing2 = bench.oracle_stratified(dag, g.n, k, budget_s=120)
        assert not missing2 and 0 < sampled2 <= eligible and est2 >= 0.0 and se2 >= 0.0


def test_alone_summary_splits_the_light_requests():
    from types import SimpleNamespace as NS

    pool = [NS(graph=NS(arcs=a)) for a in (10, 20, 5_000_000, 30)]
    out = bench._alone_summary(pool, [1.0, 2.0, 500.0, 3.0], heavy_arcs=1 << 22)
    assert out["light_p99"] < 3.01 and out["p99"] > 400 and abs(out["sum_s"] - 0.506) < 1e-9
    assert "light_p99" in bench._alone_summary(pool, [1.0, 2.0, 500.0, 3.0], heavy_arcs=0)
