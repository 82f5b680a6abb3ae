"""Host logic of the indicator workflow on CPU (no GPU): the decision
threshold keeps the requested recall of the troubled class, the confusion
counts partition the samples, the class weights balance the two classes
(each contributes half of the loss weight), and the fixed-error comparison's
history error measure."""
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


def test_history_error_columns_and_the_dilatational_floor():
    """Relative history errors per column (KE, eps_s, eps_d), the worst over
    the history; eps_d is measured against max(|eps_d|, 1e-3 |eps_s|), so at a
    vanishing eps_d (low Mach number) the error is relative to eps_s's scale."""
    ref = np.array([[1.0, 2.0, 0.5], [0.9, 4.0, 1e-9], [0.8, 8.0, 0.25]])
    h = ref.copy()
    h[0, 0] *= 1 + 3e-5          # KE off by 3e-5 at the first record
    h[2, 1] *= 1 - 2e-5          # eps_s off by 2e-5 at the last
    h[1, 2] = 1e-9 + 4e-4 * 1e-3 * 4.0  # eps_d off by 4e-4 of the floor 1e-3 eps_s
    h[2, 2] *= 1 + 1e-6
    e = gate.history_error(h, ref)
    assert np.allclose(e, [3e-5, 2e-5, 4e-4], rtol=1e-9, atol=0)
    # where eps_d is above the floor it is an ordinary relative error
    h2 = ref.copy()
    h2[0, 2] *= 1 + 7e-5
    assert np.isclose(gate.history_error(h2, ref)[2], 7e-5, rtol=1e-9)
    # identical histories: no error
    assert gate.history_error(ref, ref) == [0.0, 0.0, 0.0]
