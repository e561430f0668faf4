"""The paper-style study on the GPU path (small Monte Carlo): the proposed method saves more
operations as eta falls, and loses a few percent of sum-rate at most."""
import pytest

from paper_2512_16543_gb300 import experiment

pytestmark = pytest.mark.gpu


def test_paper_style_sweep_trends():
    res = experiment.run(batch=8, steps=80, etas=(0.9, 0.65), seed=4)
    full, e90, e65 = res["table"]
    assert full["savings_pct"] == 0.0 and full["sr_degradation_pct"] == 0.0
    assert e65["savings_pct"] >= e90["savings_pct"] > 0.0
    assert e90["mean_rank"] is not None and e90["mean_rank"] <= res["K"] / 2
    for row in (e90, e65):
        assert -1.0 < row["sr_degradation_pct"] < 15.0
        q = list(row["ecdf_quantiles"].values())
        assert q == sorted(q)
