"""What the trained controller gains over the alpha/beta rule: trained on the
GPU from record_both timings of small Kronecker graphs, scored by regret
(time of the chosen direction minus the faster one, summed over levels) on
a held-out graph of a trained size, both controllers scored on the same
recorded per-level times."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402
from paper_2012_10026_gb300 import train_controller as tc  # noqa: E402


def test_trained_controller_beats_the_rule_on_held_out_graph():
    runs = []
    for scale, seed in ((18, 11), (19, 12), (20, 13)):
        rows, nb = tc.collect(scale, seed, 10, seed + 100)
        runs += [(st, nb) for st in rows]
    X, Y, meta = tc.dataset(runs)
    assert len(X) > 50
    p, losses = tc.train(X, Y, steps=3000)
    assert losses[-1] < 0.1 * losses[0]
    rows, nb = tc.collect(20, 97, 10, 98)
    Xh, _, mh = tc.dataset([(st, nb) for st in rows])
    o0 = g3.g3_mlp_forward(p, torch.from_numpy(Xh).cuda()).cpu().numpy()[:, 0]
    r_learned = tc.regret(mh, o0 < 0)
    r_rule = tc.regret(mh, [d == 1 for (_, _, d) in mh])
    assert r_rule > 0
    assert r_learned < 0.5 * r_rule, (r_learned, r_rule)
    # with the margin past every output the rule decides every level
    assert tc.regret(mh, tc.gated(o0, mh, 1e9)) == pytest.approx(r_rule)
