"""What the trained controller gains over the alpha/beta rule: trained on the
GPU from record_both timings of small Kronecker graphs, its margin chosen
on a validation graph, and scored by regret (time of the chosen direction
minus the faster one, summed over levels) on held-out graphs of trained
sizes, both controllers scored on the same recorded per-level times."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_10026_gb300 as g3  # noqa: E402
from paper_2012_10026_gb300 import train_controller as tc  # noqa: E402


def _samples(graphs, roots=10):
    runs = []
    for scale, seed in graphs:
        rows, nb = tc.collect(scale, seed, roots, seed + 100)
        runs += [(st, nb) for st in rows]
    return tc.dataset(runs)


def _out0(p, X):
    return g3.g3_mlp_forward(p, torch.from_numpy(X).cuda()).cpu().numpy()[:, 0]


def test_trained_controller_beats_the_rule_on_held_out_graphs():
    X, Y, meta = _samples([(18, 11), (19, 12), (20, 13)])
    assert len(X) > 50
    p, losses = tc.train(X, Y, steps=3000)
    assert losses[-1] < 0.1 * losses[0]
    rule = lambda meta: [m[2] == 1 for m in meta]  # noqa: E731
    # on the graphs it was trained on, its own choices cut the rule's regret
    r_fit, r_rule_fit = tc.regret(meta, _out0(p, X) < 0), tc.regret(meta, rule(meta))
    assert r_rule_fit > 0 and r_fit < 0.5 * r_rule_fit, (r_fit, r_rule_fit)
    # margin from a validation graph, then graphs it has never seen
    Xv, _, mv = _samples([(20, 97)])
    ov = _out0(p, Xv)
    margin = tc.pick_margin({str(m): tc.regret(mv, tc.gated(ov, mv, m)) for m in tc.MARGINS})
    Xt, _, mt = _samples([(19, 98), (20, 99)])
    ot = _out0(p, Xt)
    r_learned = tc.regret(mt, tc.gated(ot, mt, margin))
    r_rule = tc.regret(mt, rule(mt))
    assert r_learned <= r_rule + 1e-6, (r_learned, r_rule, margin)
    # with the margin past every output the rule decides every level
    assert tc.regret(mt, tc.gated(ot, mt, 1e9)) == pytest.approx(r_rule)
