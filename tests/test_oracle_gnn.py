"""Pins of the warm-start network oracle (oracle/gnn.py)."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import Oracle, gnn, superop
from paper_2003_04930_gb300 import graphs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(seed, scale=0.2):
    return np.random.default_rng(seed).standard_normal(gnn.param_count()) * scale


def test_param_count():
    assert gnn.param_count() == 2 * 8 * 64 + 64 + 3 * (2 * 64 * 64 + 64) + 64 + 1 == 25921


def test_bf16_rounding_matches_library_conversion():
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 10.0 ** np.random.default_rng(1).integers(-8, 8, 10000)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(gnn.round_bf16(x), ref)
    assert gnn.round_bf16(np.float32(1.0 + 2 ** -8)) == 1.0  # tie to even
    assert gnn.round_bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6


def test_features_of_hand_worked_graph():
    with open(os.path.join(GOLDEN, "operators_n4.json")) as f:
        gd = json.load(f)
    e = np.array(gd["edges_src_dst_w"])
    A = gnn.adjacency(4, e[:, 0].astype(int), e[:, 1].astype(int), e[:, 2])
    np.testing.assert_array_equal(A, np.array(gd["A"]))
    x = gnn.features(A, 0.3, 0.85)
    np.testing.assert_allclose(x[:, 2], np.log1p([0.5, 3, 2, 0]))       # in-strength (row sums)
    np.testing.assert_allclose(x[:, 3], np.log1p(gd["outdeg"]))          # out-strength
    np.testing.assert_allclose(x[:, 4], np.log1p([1, 1, 2, 0]))
    np.testing.assert_allclose(x[:, 5], np.log1p([2, 1, 1, 0]))
    np.testing.assert_array_equal(x[:, 7], [0, 0, 0, 1])
    G = np.array(gd["G_dangling_F"])
    pi = superop.stationary_by_power_iteration(G)
    np.testing.assert_allclose(x[:, 6], np.log(4 * pi), atol=1e-12)


def _hand_params(gd):
    d = {name: np.zeros(shp) for name, shp in gnn.param_shapes()}
    for name, i, j, v in gd["weights_nonzero"]:
        if j is None:
            d[name][i] = v
        else:
            d[name][i, j] = v
    return gnn.pack(d)


def test_aggregation_and_forward_of_hand_worked_network():
    # the network definition worked out by hand on the four-node graph: the
    # aggregation matrix (built from A + A^T, rows normalised, not symmetric),
    # the first layer's pre-activations and activations, a second-layer unit
    # fed only by P h1, and the logits of the readout
    with open(os.path.join(GOLDEN, "gnn_n4.json")) as f:
        gd = json.load(f)
    A = np.array(gd["A"], dtype=np.float64)
    P = gnn.aggregation(A)
    np.testing.assert_allclose(P, np.array(gd["P"]), rtol=0, atol=1e-15)
    x = np.zeros((4, gnn.F_IN))
    x[:, :2] = np.array(gd["x_columns_0_1"], dtype=np.float64)
    th = _hand_params(gd)
    for bf16 in (True, False):  # powers of two: BF16 rounding changes nothing
        s, ph, cache = gnn.forward(th, x, P, bf16=bf16)
        h0, m1, z1 = cache[0]
        np.testing.assert_allclose(m1[:, 1], gd["layer1"]["P_v"], atol=1e-15)
        np.testing.assert_allclose(m1[:, 0], gd["layer1"]["P_ones"], atol=1e-15)
        np.testing.assert_allclose(z1[:, :3], np.array(gd["layer1"]["z_units_0_1_2"]), atol=1e-15)
        assert np.all(z1[:, 3:] == 0)
        h1 = cache[1][0]
        np.testing.assert_allclose(h1[:, :3], np.array(gd["layer1"]["h_units_0_1_2"]), atol=1e-15)
        z2 = cache[1][2]
        np.testing.assert_allclose(z2[:, 3], gd["layer2_unit3"], atol=1e-15)
        np.testing.assert_allclose(s, gd["logits"], atol=1e-14)
        # softmax of the logits: equal logits give equal probabilities, and
        # the ratio of two is exp of their difference
        assert ph[0] == pytest.approx(ph[3], rel=1e-15)
        assert ph[0] / ph[1] == pytest.approx(np.exp(2.25), rel=1e-14)
        assert ph[2] / ph[1] == pytest.approx(np.exp(1.25), rel=1e-14)


def test_pagerank_feature_equals_omega1_steady_state():
    g = graphs.heavy_tailed(30, 4)
    A = gnn.adjacency(g.n, g.src, g.dst, g.w)
    x = gnn.features(A, 1.0, 0.85)
    o = Oracle.from_edges(g, alpha=0.85, omega=1.0)
    y, steps, r, st = o.steady_state(graphs.maximally_mixed(30), 0.01, 1e-12, 200000)
    np.testing.assert_allclose(np.exp(x[:, 6]) / 30, np.real(np.diag(y)), atol=1e-11)


def test_analytic_gradient_matches_finite_differences():
    g = graphs.heavy_tailed(12, 3)
    A = gnn.adjacency(g.n, g.src, g.dst, g.w)
    x = gnn.features(A, 0.6, 0.85)
    P = gnn.aggregation(A)
    p = np.random.default_rng(2).random(12)
    p /= p.sum()
    th = _params(5)
    s, ph, cache = gnn.forward(th, x, P, bf16=False)
    grad = gnn.backward(th, P, ph, p, cache, bf16=False)
    rng = np.random.default_rng(9)
    idx = np.concatenate([rng.choice(gnn.param_count(), 60, replace=False), [gnn.param_count() - 1]])
    for i in idx:
        e = np.zeros_like(th)
        e[i] = 1e-6
        lp = gnn.loss(gnn.forward(th + e, x, P, bf16=False)[1], p)
        lm = gnn.loss(gnn.forward(th - e, x, P, bf16=False)[1], p)
        fd = (lp - lm) / 2e-6
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_softmax_loss_properties_and_equivariance():
    g = graphs.heavy_tailed(20, 8)
    th = _params(1)
    A = gnn.adjacency(g.n, g.src, g.dst, g.w)
    x, P = gnn.features(A, 0.4, 0.85), gnn.aggregation(A)
    s, ph, _ = gnn.forward(th, x, P)
    assert abs(ph.sum() - 1.0) < 1e-14 and ph.min() > 0
    p = np.random.default_rng(3).random(20)
    p /= p.sum()
    entropy = -np.sum(p * np.log(p))
    assert gnn.loss(ph, p) >= entropy - 1e-12  # Gibbs: cross-entropy >= entropy
    perm = np.random.default_rng(4).permutation(20)
    inv = np.argsort(perm)
    src, dst = inv[g.src], inv[g.dst]  # node k -> inv[k]
    A2 = gnn.adjacency(20, src, dst, g.w)
    _, ph2, _ = gnn.forward(th, gnn.features(A2, 0.4, 0.85), gnn.aggregation(A2))
    np.testing.assert_allclose(ph2[inv], ph, atol=1e-14)


def test_shipped_network_parameters_have_the_oracle_layout():
    import os
    from paper_2003_04930_gb300 import warmstart
    assert os.path.exists(warmstart.TRAINED_PARAMS)
    th = np.load(warmstart.TRAINED_PARAMS)
    assert th.dtype == np.float32 and th.shape == (gnn.param_count(),)
    assert np.all(np.isfinite(th))
