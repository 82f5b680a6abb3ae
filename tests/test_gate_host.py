"""Host logic of the indicator workflow on CPU (no GPU): the decision
threshold keeps the requested recall of the troubled class, the confusion
counts partition the samples, and the class weights balance the two classes
(each contributes half of the loss weight)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_07387_gb300 import gate


class _Logits:
    """Stands in for the network: returns fixed logits."""

    def __init__(self, z):
        self.z = z

    def forward(self, X):
        return self.z


def _data(n=20000, seed=0):
    rng = np.random.default_rng(seed)
    z = torch.tensor(rng.normal(size=n), dtype=torch.float32)
    y = ((z + torch.tensor(0.7 * rng.normal(size=n), dtype=torch.float32)) > 1.8).float()
    return z, y


@pytest.mark.parametrize("recall", [0.9, 0.99, 0.999, 1.0])
def test_threshold_keeps_the_recall(recall):
    z, y = _data()
    net = _Logits(z)
    thr = gate.threshold_for_recall(net, None, y, recall)
    c = gate.confusion(net, None, y, thr)
    assert c["recall"] >= recall
    assert c["tp"] + c["fn"] + c["fp"] + c["tn"] == z.numel()
    assert c["tp"] + c["fn"] == int(y.sum().item())
    # the threshold does not flag more than needed: just above the lowest
    # troubled logit that it keeps, recall would fall below the target
    zp = z[y > 0.5]
    kept = zp[zp > thr]
    worse = gate.confusion(net, None, y, float(kept.min().item()))
    assert worse["recall"] < recall or kept.numel() == zp.numel() and recall == 1.0 and worse["recall"] < 1.0


def test_threshold_without_troubled_samples_flags_nothing():
    z = torch.zeros(100)
    assert gate.threshold_for_recall(_Logits(z), None, torch.zeros(100), 0.999) == float("inf")


def test_class_weights_balance_the_classes():
    _, y = _data()
    w_pos, w_neg = gate.class_weights(y)
    p = float(y.mean().item())
    assert abs(w_pos * p - 0.5) < 1e-12 and abs(w_neg * (1 - p) - 0.5) < 1e-12
