"""What the trained controller gains over the alpha/beta rule, by the same
protocol as train_controller.py: trained on the GPU from record_both timings
of Kronecker graphs at SCALE 20-24, its margin chosen on a held-out SCALE 24
graph, and scored by regret (time of the chosen direction minus the faster
one, summed over levels) on a SCALE 25 graph it has never seen, both
controllers scored on the same recorded per-level times."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402
from paper_2012_10026_gb300 import train_controller as tc  # noqa: E402


def _samples(graphs, roots):
    runs = []
    for scale, seed in graphs:
        rows, nb = tc.collect(scale, seed, roots, seed + 100)
        runs += [(st, nb) for st in rows]
    return tc.dataset(runs)


def _out0(p, X):
    return g3.g3_mlp_forward(p, torch.from_numpy(X).cuda()).cpu().numpy()[:, 0]


def test_trained_controller_beats_the_rule_on_a_larger_unseen_graph():
    X, Y, meta = _samples([(20, 11), (21, 12), (22, 13), (23, 14), (24, 15)], 12)
    assert len(X) > 200
    p, losses = tc.train(X, Y, steps=3000)
    assert losses[-1] < 0.1 * losses[0]
    rule = lambda meta: [m[2] == 1 for m in meta]  # noqa: E731
    o_fit = _out0(p, X)
    r_fit, r_rule_fit = tc.regret(meta, o_fit < 0), tc.regret(meta, rule(meta))
    # margin from a held-out graph of the largest trained size
    Xv, _, mv = _samples([(24, 97)], 12)
    ov = _out0(p, Xv)
    table = {str(m): tc.regret(mv, tc.gated(ov, mv, m)) for m in tc.MARGINS}
    margin = tc.pick_margin(table)
    # a graph twice the largest trained size, never seen
    Xt, _, mt = _samples([(25, 98)], 16)
    ot = _out0(p, Xt)
    r_learned = tc.regret(mt, tc.gated(ot, mt, margin))
    r_rule = tc.regret(mt, rule(mt))
    # on the graphs it was trained on, its own choices beat the rule's
    assert r_rule_fit > 0 and r_fit < r_rule_fit, (r_fit, r_rule_fit)
    assert r_learned <= r_rule + 1e-6, (r_learned, r_rule, margin)
    # with the margin past every output the rule decides every level
    assert tc.regret(mt, tc.gated(ot, mt, 1e9)) == pytest.approx(r_rule)
