"""Host-side logic of the learned form's training driver (no GPU): the
weights file, the validation rule that decides what ships, and the constant
policies used to label the shift head."""
import numpy as np

from oracle import mlp_ref as M


def _learn():
    from paper_2404_09276_gb300 import learn

    return learn


def test_committed_weights_load_and_ship_flag(tmp_path):
    learn = _learn()
    w, ship = learn.load_weights()
    assert w is not None and w.shape == (M.N_PARAMS,) and np.all(np.isfinite(w))
    assert ship  # the committed file passed its validation
    p = tmp_path / "w.txt"
    p.write_text("# ship: plain\n" + "\n".join("0.5" for _ in range(M.N_PARAMS)) + "\n")
    w2, ship2 = learn.load_weights(str(p))
    assert not ship2 and np.all(w2 == 0.5)
    p.write_text("# ship: learned\n1.0\n2.0\n")  # wrong length
    assert learn.load_weights(str(p))[0] is None
    assert learn.load_weights(str(tmp_path / "missing.txt")) == (None, False)


def test_validation_rule_counts_only_learned_misses():
    """A learned run fails only where it exceeds tol and the plain rule's run
    on the same matrix meets it (R11)."""
    learn = _learn()
    tol = learn.TOL
    rows = [
        dict(seed=1, plain_passes=6, learned_passes=5, plain_s=1.0, learned_s=0.8, plain_eps=0.5 * tol, learned_eps=0.9 * tol),
        dict(seed=2, plain_passes=6, learned_passes=4, plain_s=1.0, learned_s=0.7, plain_eps=0.5 * tol, learned_eps=1.5 * tol),
        dict(seed=3, plain_passes=7, learned_passes=5, plain_s=1.2, learned_s=0.9, plain_eps=2.0 * tol, learned_eps=3.0 * tol),
        dict(seed=4, plain_passes=5, learned_passes=5, plain_s=0.9, learned_s=0.9, plain_eps=1.5 * tol, learned_eps=0.5 * tol),
    ]
    s = learn.summarize(rows)
    assert s["failures"] == 1 and s["fail_seeds"][0][0] == 2
    assert s["plain_failures"] == 2 and s["both_over"] == 1
    assert s["plain_passes"] == 6.0 and s["learned_passes"] == 4.75
    assert abs(s["learned_s"] - 3.3) < 1e-12


def test_constant_policies():
    """_const_net(o0, o1) is the zero network with output biases (o0, o1), and
    _logit(f) the bias whose sigmoid is f (f = 1 saturates: sigmoid(40) is 1 in FP32)."""
    learn = _learn()
    for f in learn.FRACTIONS:
        w = learn._const_net(learn._logit(f), -40.0)
        _, o = M.forward(w.astype(np.float64), np.random.default_rng(0).uniform(-3, 3, (5, M.N_IN)))
        sig = 1 / (1 + np.exp(-o[:, 0]))
        assert np.allclose(sig, f, atol=1e-12 if f < 1 else 1e-17)
        assert np.all(o[:, 1] == -40.0)
    assert np.float32(1 / (1 + np.exp(-np.float32(40.0)))) == np.float32(1.0)
