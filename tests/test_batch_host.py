"""Host logic of the batched sweep's campaign re-tuning (paper_1805_07251_gb300.batch),
checked on the CPU with a stand-in for the GPU batch: which runs are re-tuned, how often,
and with which parameters."""
import numpy as np
import pytest

from paper_1805_07251_gb300 import batch as B


class FakeBatch:
    """Stands in for Batch: a run 'fails' while its kappa scale is below its need."""

    need = {}
    created = []

    def __init__(self, runs, *a, **kw):
        self.runs = [dict(r) for r in runs]
        FakeBatch.created.append([r["id"] for r in runs])

    def init(self, fields):
        assert len(fields) == len(self.runs)

    def step(self, n):
        pass

    def errors(self):
        return np.array([1 if r.get("kappa_scale", 1.0) < FakeBatch.need.get(r["id"], 1.0) else 0 for r in self.runs])

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(B, "Batch", FakeBatch)
    FakeBatch.created = []
    return FakeBatch


def runs(k):
    return [dict(id=i, lattice="D1Q3", nx=64, ny=1, kT=0.5, gamma_mu=0.08) for i in range(k)]


def test_retune_widens_interfaces_and_lowers_gamma():
    r = B.retune(dict(gamma_mu=0.08))
    assert r["kappa_scale"] == B.KAPPA_STEP and r["gamma_mu"] == 0.08 / B.KAPPA_STEP
    assert r["width"] == 2.0 * B.KAPPA_STEP ** 0.5 and r["retuned"] == 1
    r2 = B.retune(r)
    assert r2["kappa_scale"] == B.KAPPA_STEP ** 2 and r2["retuned"] == 2


def test_prescan_retunes_only_failing_runs(fake):
    fake.need = {1: 4.0, 3: 16.0, 4: 1e9}
    recs, still = B.prescan(runs(6), lambda r: np.zeros(1), None, None, None, None, 2, rounds=2)
    assert [r.get("retuned", 0) for r in recs] == [0, 1, 0, 2, 2, 0]
    assert recs[1]["kappa_scale"] == 4.0 and recs[3]["kappa_scale"] == 16.0
    assert still == 1                      # run 4 still fails after two re-tunings
    # the first scan covers every run, later scans only the runs that failed
    assert fake.created == [[0, 1, 2, 3, 4, 5], [1, 3, 4], [3, 4]]


def test_prescan_without_failures_scans_once(fake):
    fake.need = {}
    recs, still = B.prescan(runs(3), lambda r: np.zeros(1), None, None, None, None, 2)
    assert still == 0 and all("retuned" not in r for r in recs) and len(fake.created) == 1
