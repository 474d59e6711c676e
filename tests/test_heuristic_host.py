"""Host-side steps of the learned heuristic's training pipeline (no GPU): the
standardisation folded into the first layer gives, on raw features, the
logit the trained network gives on standardised ones; fit() passes the
standardised samples to the device trainer and returns folded weights; the
static features are those a rule has before the first decision."""
import numpy as np

from paper_1909_01786_gb300 import aspgpu, heuristic


def test_folded_weights_give_the_same_logit_on_raw_features():
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.5, aspgpu.MLP_PARAMS).astype(np.float32)
    X = rng.normal(3.0, 2.0, (500, heuristic.N_FEATURES)).astype(np.float32)
    mu, sd = X.mean(0), X.std(0)
    folded = heuristic.fold_standardisation(w, mu, sd)
    want = heuristic.forward_np(w, (X - mu) / sd)
    got = heuristic.forward_np(folded, X)
    assert np.allclose(got, want, rtol=1e-4, atol=1e-4)
    # the second layer is untouched
    W1, b1, w2, b2 = heuristic.split(folded)
    assert np.array_equal(w2, heuristic.split(w)[2]) and np.array_equal(b2, heuristic.split(w)[3])


def test_fit_trains_on_standardised_samples_and_folds(monkeypatch):
    rng = np.random.default_rng(1)
    X = rng.normal(1.0, 3.0, (256, heuristic.N_FEATURES)).astype(np.float32)
    X[:, 7] = 1.0                                   # a constant feature keeps sd = 1
    y = (rng.random(256) < 0.5).astype(np.float32)
    trained = rng.normal(0, 0.3, aspgpu.MLP_PARAMS).astype(np.float32)
    seen = {}

    def fake_train(Z, labels, w0, epochs, learning_rate):
        seen["Z"], seen["y"] = Z.copy(), labels.copy()
        return trained.copy()

    monkeypatch.setattr(aspgpu, "train_mlp", fake_train)
    out, stats = heuristic.fit(X, y, epochs=3)
    Z = seen["Z"]
    assert np.allclose(Z[:, :7].mean(0), 0, atol=1e-4) and np.allclose(Z[:, :7].std(0), 1, atol=1e-3)
    assert np.allclose(Z[:, 7], 0)
    assert np.array_equal(seen["y"], y)
    assert np.allclose(heuristic.forward_np(out, X), heuristic.forward_np(trained, Z), rtol=1e-4, atol=1e-4)
    assert stats["samples"] == 256 and 0.0 <= stats["train_accuracy"] <= 1.0


def test_static_features_are_the_values_before_the_first_decision():
    rng = np.random.default_rng(2)
    X = rng.random((10, heuristic.N_FEATURES)).astype(np.float32)
    Z = heuristic.static_features(X)
    assert np.array_equal(Z[:, :8], X[:, :8])
    assert np.array_equal(Z[:, 9], X[:, 2])
    assert (Z[:, 8] == 0).all() and (Z[:, 10] == 0).all() and (Z[:, 12:] == 0).all()
    assert np.allclose(Z[:, 11], 1.0 / 64.0)
